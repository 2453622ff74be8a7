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

// sum over the 2^k lanes of an aligned group (xor butterfly); every lane of
// the group ends with the same pair (two_sum is symmetric in its arguments)
__device__ __forceinline__ float2 df_xor_add(float2 v, int o) {
    const float oh = __shfl_xor_sync(0xffffffffu, v.x, o), ol = __shfl_xor_sync(0xffffffffu, v.y, o);
    return df_add(v, make_float2(oh, ol));
}

}  // namespace rfm
