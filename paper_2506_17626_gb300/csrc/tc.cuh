// tc.cuh -- tcgen05 building blocks shared by the tensor-core products of the
// many-right-hand-side LSQR: BF16 x BF16 -> FP32 MMAs (kind::f16) with
// operands in shared memory in the canonical K-major layout without swizzle
// (8 x 8 BF16 core matrices of 128 contiguous bytes, rows of 16 bytes; the
// next core matrix along K 128 bytes on, the next 8 rows KC / 8 core
// matrices on) and the accumulator in tensor memory.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace rfm {

__device__ inline unsigned tcm_su32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) of a K-major operand whose K extent is KC
template <int KC>
__device__ inline int tcm_off(int r, int k) {
    return ((r >> 3) * (KC / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// shared-memory descriptor of a K-major operand (K extent KC) starting at base
template <int KC>
__device__ inline uint64_t tcm_desc(const void *base) {
    uint64_t d = (uint64_t)((tcm_su32(base) >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;              // leading byte offset: next core matrix along K
    d |= (uint64_t)((KC / 8 * 128) >> 4) << 32;   // stride byte offset: next 8 rows
    d |= (uint64_t)1 << 46;                       // descriptor version
    return d;                                     // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: BF16 A and B (K-major), FP32 D, M x N
__host__ __device__ constexpr uint32_t tcm_idesc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ inline void tcm_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

__device__ inline void tcm_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(tcm_su32(mbar)) : "memory");
}

// bounded wait on an mbarrier phase (false after about 2^26 tries)
__device__ inline bool tcm_wait(uint64_t *mbar, unsigned parity) {
    for (long it = 0; it < (1l << 26); ++it) {
        unsigned d;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(d) : "r"(tcm_su32(mbar)), "r"(parity) : "memory");
        if (d) return true;
    }
    return false;
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes
__device__ inline void tcm_ld32(uint32_t addr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes
__device__ inline void tcm_ld16(uint32_t addr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// x = h0 + h1 + h2 in BF16 (each the rounding of what the previous terms
// leave), 24 significant bits in all: the FP32 value to within about
// 2^-24 |x|.  Products of two split values keep the six terms whose orders
// add up to at most 2; the three dropped ones are below 2^-24 |x y|.
__device__ inline void bf16_split3(float x, __nv_bfloat16 &h0, __nv_bfloat16 &h1, __nv_bfloat16 &h2) {
    h0 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h0);
    h1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(h1);
    h2 = __float2bfloat16_rn(r2);
}

// bf16_split3 of two values at once (packed conversions, the same rounding):
// the three terms as bf16x2 words, x[0] in the low half (the lower address)
__device__ inline void bf16_split3x2(float a, float b, uint32_t &w0, uint32_t &w1, uint32_t &w2) {
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(a, b);
    const float2 f0 = __bfloat1622float2(h0);
    const float ra = a - f0.x, rb = b - f0.y;
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(ra, rb);
    const float2 f1 = __bfloat1622float2(h1);
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(ra - f1.x, rb - f1.y);
    w0 = *reinterpret_cast<const uint32_t *>(&h0);
    w1 = *reinterpret_cast<const uint32_t *>(&h1);
    w2 = *reinterpret_cast<const uint32_t *>(&h2);
}

// 8 consecutive-K values of one row, split, stored as 16-byte core-matrix
// rows into the three split operands (byte offset off, split stride sz)
__device__ inline void tcm_store8(unsigned char *base, int off, int sz, const float (&x)[8]) {
    uint4 w[3];
    bf16_split3x2(x[0], x[1], w[0].x, w[1].x, w[2].x);
    bf16_split3x2(x[2], x[3], w[0].y, w[1].y, w[2].y);
    bf16_split3x2(x[4], x[5], w[0].z, w[1].z, w[2].z);
    bf16_split3x2(x[6], x[7], w[0].w, w[1].w, w[2].w);
#pragma unroll
    for (int s = 0; s < 3; ++s) *reinterpret_cast<uint4 *>(base + s * sz + off) = w[s];
}

}  // namespace rfm
