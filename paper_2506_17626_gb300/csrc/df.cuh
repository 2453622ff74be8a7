// df.cuh -- double-float arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum h + l of two floats, |l| <= ulp(h) (Dekker,
// "A floating-point technique for extending the available precision",
// Numer. Math. 18, 1971), which carries about 48 significant bits.  The
// error-free transformations are Knuth's two-sum (TAOCP vol. 2, 4.2.2,
// Theorem B) and the FMA two-product (the exact error of a * b is
// fma(a, b, -a * b)).  GB300 issues FP32 instructions at 64 times its FP64
// rate, so a double-float multiply-add (about a dozen FP32 instructions)
// costs a fraction of one FP64 instruction.
//
// Every operation goes through the _rn intrinsics, which the compiler never
// contracts into FMAs: contraction would break the error terms.
#pragma once

#include <cuda_runtime.h>

namespace rfm {

// s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e == a + b exactly, given |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ float2 df_from_double(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ double df_to_double(float2 a) { return (double)a.x + (double)a.y; }

__device__ __forceinline__ float df_to_float(float2 a) { return __fadd_rn(a.x, a.y); }

// a + b, normalised
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    float h, l;
    fast_two_sum(s, e, h, l);
    return make_float2(h, l);
}

__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ float2 df_sub(float2 a, float2 b) { return df_add(a, df_neg(b)); }

// a * b, normalised (the l * l term is below the format's precision)
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    float h, l;
    fast_two_sum(p, e, h, l);
    return make_float2(h, l);
}

// (sh, sl) += a * b.  The accumulator is left unnormalised: sl collects the
// error terms of the running sum (it stays far below sh), and the pair is
// normalised when it is read out.
__device__ __forceinline__ void df_acc(float2 a, float2 b, float &sh, float &sl) {
    const float p = __fmul_rn(a.x, b.x);
    float pe = __fmaf_rn(a.x, b.x, -p);
    pe = __fmaf_rn(a.x, b.y, pe);
    pe = __fmaf_rn(a.y, b.x, pe);
    float s, e;
    two_sum(sh, p, s, e);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(e, pe));
}

// a - e * x, normalised
__device__ __forceinline__ float2 df_axmy(float2 a, float2 e, float2 x) {
    const float p = __fmul_rn(e.x, x.x);
    float pe = __fmaf_rn(e.x, x.x, -p);
    pe = __fmaf_rn(e.x, x.y, pe);
    pe = __fmaf_rn(e.y, x.x, pe);
    float s, t;
    two_sum(a.x, -p, s, t);
    t = __fadd_rn(t, __fsub_rn(a.y, pe));
    float h, l;
    fast_two_sum(s, t, h, l);
    return make_float2(h, l);
}

// sqrt(a) for a > 0: the FP32 root y, then one Newton (Heron) step carried
// out in double-float, y + (a - y^2) / (2 y), with y^2 formed exactly (the
// double-length square root of Dekker 1971)
__device__ __forceinline__ float2 df_sqrt(float2 a) {
    const float y = __fsqrt_rn(a.x);
    const float p = __fmul_rn(y, y);
    const float pe = __fmaf_rn(y, y, -p);
    const float r = __fadd_rn(__fsub_rn(a.x, p), __fsub_rn(a.y, pe));
    float h, l;
    fast_two_sum(y, __fdiv_rn(r, __fmul_rn(2.f, y)), h, l);
    return make_float2(h, l);
}

// 1 / a for a != 0: the FP32 reciprocal y, then one Newton step
// y + y (1 - a y) with the residual 1 - a y formed to double-float accuracy
__device__ __forceinline__ float2 df_rcp(float2 a) {
    const float y = __frcp_rn(a.x);
    const float p = __fmul_rn(a.x, y);
    const float pe = __fmaf_rn(a.x, y, -p);
    float r = __fsub_rn(__fsub_rn(1.f, p), pe);
    r = __fmaf_rn(-a.y, y, r);
    float h, l;
    fast_two_sum(y, __fmul_rn(y, r), h, l);
    return make_float2(h, l);
}

// a * 2^k for integer k (both words scaled exactly, no overflow in range)
__device__ __forceinline__ float2 df_ldexp(float2 a, int k) { return make_float2(ldexpf(a.x, k), ldexpf(a.y, k)); }

// Double-float constant from a double known at compile time.
struct DfConst {
    float h, l;
    constexpr DfConst(double x) : h((float)x), l((float)(x - (double)(float)x)) {}
};

// expm1(r) = sum_{n >= 1} r^n / n! for |r| <= ln2 / 2, by Horner's rule
// on the Taylor series cut after n = 13 (the next term is below 2^-52 of
// the sum there).
__device__ __forceinline__ float2 df_expm1_reduced(float2 r) {
    constexpr double f[14] = {1.0, 1.0, 1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040,
                              1.0 / 40320, 1.0 / 362880, 1.0 / 3628800, 1.0 / 39916800, 1.0 / 479001600,
                              1.0 / 6227020800.0};
    float2 p = make_float2(DfConst(f[13]).h, DfConst(f[13]).l);
#pragma unroll
    for (int n = 12; n >= 1; --n) p = df_add(df_mul(p, r), make_float2(DfConst(f[n]).h, DfConst(f[n]).l));
    return df_mul(p, r);
}

// tanh(z) in double-float.  With x = 2|z|: for x <= ln2/2, tanh = e / (e + 2)
// with e = expm1(x) (no cancellation near 0); otherwise x = k ln2 + r with
// |r| <= ln2/2, E = 2^k (1 + expm1(r)) = exp(x) and tanh = 1 - 2 / (E + 1);
// |z| > 20 gives 1 (tanh(20) = 1 - 8.5e-18).  The sign follows z.
__device__ __forceinline__ float2 df_tanh(float2 z) {
    const bool neg = z.x < 0.f;
    const float2 az = neg ? df_neg(z) : z;
    float2 t;
    if (az.x > 20.f) {
        t = make_float2(1.f, 0.f);
    } else {
        const float2 x = make_float2(2.f * az.x, 2.f * az.y);
        constexpr double kLn2 = 0.693147180559945309417232121458;
        if (x.x <= 0.34657359f) {
            const float2 e = df_expm1_reduced(x);
            t = df_mul(e, df_rcp(df_add(e, make_float2(2.f, 0.f))));
        } else {
            const float k = rintf(x.x * 1.44269504f);
            const float rh = __fmaf_rn(-k, DfConst(kLn2).h, x.x);   // exact: x.x and k ln2_hi agree in their leading bits
            const float2 r = df_add(make_float2(rh, 0.f), make_float2(__fmaf_rn(-k, DfConst(kLn2).l, x.y), 0.f));
            const float2 E = df_ldexp(df_add(df_expm1_reduced(r), make_float2(1.f, 0.f)), (int)k);
            const float2 q = df_rcp(df_add(E, make_float2(1.f, 0.f)));
            t = df_sub(make_float2(1.f, 0.f), make_float2(2.f * q.x, 2.f * q.y));
        }
    }
    return neg ? df_neg(t) : t;
}

// sum over the 2^k lanes of an aligned group (xor butterfly); every lane of
// the group ends with the same pair (two_sum is symmetric in its arguments)
__device__ __forceinline__ float2 df_xor_add(float2 v, int o) {
    const float oh = __shfl_xor_sync(0xffffffffu, v.x, o), ol = __shfl_xor_sync(0xffffffffu, v.y, o);
    return df_add(v, make_float2(oh, ol));
}

}  // namespace rfm
