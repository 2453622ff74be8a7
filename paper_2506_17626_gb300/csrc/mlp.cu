// mlp.cu -- the warm-start network: forward pass, loss gradient by
// backpropagation, deterministic reduction of the per-CTA gradients, Adam.
//
// Network: widths w[0..L]; layer l computes z_l = W_l h_{l-1} + b_l with
// h_l = tanh(z_l) on hidden layers and a linear scalar output.  Parameters are
// packed layer by layer, W_l row-major (w[l] x w[l-1]) then b_l, in FP32.
//
// One CTA handles tiles of kTS samples and keeps every activation of its tile
// in shared memory, so the backward pass reads nothing but the staged weights
// again.  The error of layer l-1 overwrites the activation h_{l-1} once the
// weight gradient of layer l has consumed it.  Each CTA accumulates its
// gradient over its tiles in its own slice of the workspace; a second kernel
// sums the slices in a fixed order (the result does not depend on timing).
#include <math.h>

#include <cuda_bf16.h>

#include "common.cuh"
#include "prof.cuh"

namespace rfm {

constexpr int kMlpThreads = 256;
constexpr int kTS = 64;             // samples per tile
constexpr int kMlpMaxLayers = 8;
constexpr int kMlpMaxWidth = 128;   // hidden widths: multiples of 16 up to this
constexpr int kMlpMaxIn = 32;       // input width
constexpr int kMlpMaxCtas = 512;    // gradient slices

struct MlpDesc {
    int L;
    int w[kMlpMaxLayers + 1];
    int ld[kMlpMaxLayers];           // shared-memory row stride of h_l (l < L)
    int64_t off[kMlpMaxLayers + 1];  // parameter offset of layer l (1-based)
    int64_t np;
    int hoff[kMlpMaxLayers];         // float offset of h_l in shared memory
    int woff;                        // float offset of the staged weights
    int smem_floats;
};

static rfm_status mlp_desc(const rfm_mlp *net, MlpDesc *d) {
    if (!net || net->n_layers < 1 || net->n_layers > kMlpMaxLayers) {
        set_error("rfm_mlp: n_layers must be 1..%d", kMlpMaxLayers);
        return RFM_EINVAL;
    }
    const int L = net->n_layers;
    d->L = L;
    for (int l = 0; l <= L; ++l) d->w[l] = net->width[l];
    if (d->w[0] < 1 || d->w[0] > kMlpMaxIn) {
        set_error("rfm_mlp: input width must be 1..%d", kMlpMaxIn);
        return RFM_EINVAL;
    }
    if (d->w[L] != 1) {
        set_error("rfm_mlp: the output width must be 1");
        return RFM_EINVAL;
    }
    for (int l = 1; l < L; ++l)
        if (d->w[l] < 16 || d->w[l] > kMlpMaxWidth || d->w[l] % 16) {
            set_error("rfm_mlp: hidden widths must be multiples of 16 up to %d", kMlpMaxWidth);
            return RFM_EINVAL;
        }
    int64_t o = 0;
    int maxw = 0;
    for (int l = 1; l <= L; ++l) {
        d->off[l] = o;
        o += (int64_t)d->w[l] * d->w[l - 1] + d->w[l];
        const int wsz = d->w[l] * (d->w[l - 1] + 1);
        if (wsz > maxw) maxw = wsz;
    }
    d->off[0] = 0;
    d->np = o;
    int f = 0;
    for (int l = 0; l < L; ++l) {
        // +4 floats: rows of consecutive sample groups fall on different banks
        d->ld[l] = d->w[l] + 4;
        d->hoff[l] = f;
        f += kTS * d->ld[l];
    }
    d->woff = f;
    f += maxw + kMlpMaxWidth;   // staged W (row stride w[l-1]+1) and bias
    f += 2 * kTS + 64;          // output-layer errors, reductions
    d->smem_floats = f;
    if ((size_t)f * 4 > 227 * 1024) {
        set_error("rfm_mlp: the network's activations need %d bytes of shared memory per %d samples (max %d)",
                  f * 4, kTS, 227 * 1024);
        return RFM_EINVAL;
    }
    return RFM_OK;
}

// Staged copy of W_l (row stride ni+1, so consecutive rows start on
// consecutive banks) and b_l.
__device__ inline void stage_weights(const float *__restrict__ theta, const MlpDesc &D, int l, float *sW, float *sb) {
    const int no = D.w[l], ni = D.w[l - 1];
    const float *W = theta + D.off[l];
    for (int e = threadIdx.x; e < no * ni; e += kMlpThreads) {
        const int o = e / ni, i = e - o * ni;
        sW[o * (ni + 1) + i] = __ldg(W + e);
    }
    for (int o = threadIdx.x; o < no; o += kMlpThreads) sb[o] = __ldg(W + (int64_t)no * ni + o);
}

// Hidden layer l forward for the tile: h_l = tanh(h_{l-1} W_l^T + b_l).
// Thread (sg, og): samples 4 sg .. 4 sg + 3, outputs og + 16 q.
__device__ inline void hidden_forward(const MlpDesc &D, int l, float *sm, const float *sW, const float *sb) {
    const int no = D.w[l], ni = D.w[l - 1];
    const float *H = sm + D.hoff[l - 1];
    float *Z = sm + D.hoff[l];
    const int ldh = D.ld[l - 1], ldz = D.ld[l];
    const int sg = threadIdx.x >> 4, og = threadIdx.x & 15;
    const int nq = no / 16;
    float acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[a][q] = 0.f;
    for (int k = 0; k < ni; ++k) {
        float h[4], wv[8];
#pragma unroll
        for (int a = 0; a < 4; ++a) h[a] = H[(4 * sg + a) * ldh + k];
#pragma unroll
        for (int q = 0; q < 8; ++q) wv[q] = q < nq ? sW[(og + 16 * q) * (ni + 1) + k] : 0.f;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[a][q] = fmaf(h[a], wv[q], acc[a][q]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if (q >= nq) break;
        const int o = og + 16 * q;
#pragma unroll
        for (int a = 0; a < 4; ++a) Z[(4 * sg + a) * ldz + o] = tanhf(acc[a][q] + sb[o]);
    }
}

template <bool GRAD>
__global__ void __launch_bounds__(kMlpThreads, 1)
    k_mlp(MlpDesc D, const float *__restrict__ theta, const float *__restrict__ X, const float *__restrict__ T,
          int64_t n, float *__restrict__ Y, float *__restrict__ gpart, double *__restrict__ lpart, float inv_n) {
    extern __shared__ __align__(16) float sm[];
    float *sW = sm + D.woff;
    const int L = D.L;
    float *sb = sW + (D.smem_floats - D.woff - kMlpMaxWidth - 2 * kTS - 64);   // bias after the largest W
    float *eo = sb + kMlpMaxWidth;     // output-layer error per sample (kTS)
    float *yo = eo + kTS;              // outputs of the tile (kTS)
    float *red = yo + kTS;             // 64 floats of reduction scratch
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n_tiles = (n + kTS - 1) / kTS;
    float *gmine = GRAD ? gpart + (int64_t)blockIdx.x * D.np : nullptr;
    double lsum = 0.0;
    bool first = true;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t s0 = tile * kTS;
        const int ns = (int)min((int64_t)kTS, n - s0);
        // inputs (rows beyond the batch are zero)
        {
            float *H0 = sm + D.hoff[0];
            const int ni = D.w[0], ld0 = D.ld[0];
            for (int e = tid; e < kTS * ni; e += kMlpThreads) {
                const int s = e / ni, i = e - s * ni;
                H0[s * ld0 + i] = s < ns ? __ldg(X + (s0 + s) * ni + i) : 0.f;
            }
        }
        __syncthreads();
        for (int l = 1; l < L; ++l) {
            stage_weights(theta, D, l, sW, sb);
            __syncthreads();
            hidden_forward(D, l, sm, sW, sb);
            __syncthreads();
        }
        // output layer: y = h_{L-1} . w_L + b_L, one warp per 8 samples
        {
            const int ni = D.w[L - 1], ldh = D.ld[L - 1];
            const float *H = sm + D.hoff[L - 1];
            const float *wL = theta + D.off[L];
            const float bL = __ldg(wL + ni);
            for (int s = warp; s < kTS; s += kMlpThreads / 32) {
                float t = 0.f;
                for (int i = lane; i < ni; i += 32) t = fmaf(H[s * ldh + i], __ldg(wL + i), t);
                for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                if (lane == 0) {
                    const float yv = t + bL;
                    yo[s] = yv;
                    if (!GRAD && s < ns) Y[s0 + s] = yv;
                    if (GRAD) {
                        const float d = s < ns ? yv - __ldg(T + s0 + s) : 0.f;
                        eo[s] = 2.f * d * inv_n;
                        lsum += (double)d * (double)d;
                    }
                }
            }
        }
        __syncthreads();
        if (!GRAD) continue;
        // ---- backward
        // output layer: dW_L = sum_s e_s h_{L-1,s}, db_L = sum_s e_s,
        // e_{L-1} = e_s w_L (1 - h^2) written over h_{L-1}
        {
            const int ni = D.w[L - 1], ldh = D.ld[L - 1];
            float *H = sm + D.hoff[L - 1];
            const float *wL = theta + D.off[L];
            float *g = gmine + D.off[L];
            for (int i = tid; i < ni; i += kMlpThreads) {
                float t = 0.f;
                for (int s = 0; s < kTS; ++s) t = fmaf(eo[s], H[s * ldh + i], t);
                g[i] = first ? t : g[i] + t;
            }
            if (warp == 0) {
                float t = 0.f;
                for (int s = lane; s < kTS; s += 32) t += eo[s];
                for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                if (lane == 0) g[ni] = first ? t : g[ni] + t;
            }
            __syncthreads();
            if (L > 1)
                for (int e = tid; e < kTS * ni; e += kMlpThreads) {
                    const int s = e / ni, i = e - s * ni;
                    const float h = H[s * ldh + i];
                    H[s * ldh + i] = eo[s] * __ldg(wL + i) * (1.f - h * h);
                }
            __syncthreads();
        }
        for (int l = L - 1; l >= 1; --l) {
            const int no = D.w[l], ni = D.w[l - 1];
            const int lde = D.ld[l], ldh = D.ld[l - 1];
            const float *E = sm + D.hoff[l];      // e_l (over h_l)
            float *H = sm + D.hoff[l - 1];        // h_{l-1}, then e_{l-1}
            float *g = gmine + D.off[l];
            // weight gradient: dW_l[o][i] = sum_s e_l[s][o] h_{l-1}[s][i]
            {
                const int og = tid & 15, ig = tid >> 4;
                const int nq = no / 16;
                const int nr = (ni + 15) / 16;
                for (int r0 = 0; r0 < nr; r0 += 8) {
                    float acc[8][8];
#pragma unroll
                    for (int q = 0; q < 8; ++q)
#pragma unroll
                        for (int r = 0; r < 8; ++r) acc[q][r] = 0.f;
                    for (int s = 0; s < kTS; ++s) {
                        float ev[8], hv[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) ev[q] = q < nq ? E[s * lde + og + 16 * q] : 0.f;
#pragma unroll
                        for (int r = 0; r < 8; ++r) {
                            const int i = ig + 16 * (r0 + r);
                            hv[r] = i < ni ? H[s * ldh + i] : 0.f;
                        }
#pragma unroll
                        for (int q = 0; q < 8; ++q)
#pragma unroll
                            for (int r = 0; r < 8; ++r) acc[q][r] = fmaf(ev[q], hv[r], acc[q][r]);
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        if (q >= nq) break;
                        const int o = og + 16 * q;
#pragma unroll
                        for (int r = 0; r < 8; ++r) {
                            const int i = ig + 16 * (r0 + r);
                            if (i < ni) {
                                float *p = g + (int64_t)o * ni + i;
                                *p = first ? acc[q][r] : *p + acc[q][r];
                            }
                        }
                    }
                }
                for (int o = tid; o < no; o += kMlpThreads) {
                    float t = 0.f;
                    for (int s = 0; s < kTS; ++s) t += E[s * lde + o];
                    float *p = g + (int64_t)no * ni + o;
                    *p = first ? t : *p + t;
                }
            }
            if (l == 1) break;
            stage_weights(theta, D, l, sW, sb);
            __syncthreads();   // also: every read of h_{l-1} for dW_l is done
            // e_{l-1}[s][i] = (sum_o e_l[s][o] W_l[o][i]) (1 - h_{l-1}[s][i]^2)
            {
                const int sg = tid >> 4, ig = tid & 15;
                const int nq = ni / 16;   // ni is a hidden width here (l >= 2)
                float acc[4][8];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int q = 0; q < 8; ++q) acc[a][q] = 0.f;
                for (int o = 0; o < no; ++o) {
                    float ev[4], wv[8];
#pragma unroll
                    for (int a = 0; a < 4; ++a) ev[a] = E[(4 * sg + a) * lde + o];
#pragma unroll
                    for (int q = 0; q < 8; ++q) wv[q] = q < nq ? sW[o * (ni + 1) + ig + 16 * q] : 0.f;
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int q = 0; q < 8; ++q) acc[a][q] = fmaf(ev[a], wv[q], acc[a][q]);
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (q >= nq) break;
                    const int i = ig + 16 * q;
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        float *p = H + (4 * sg + a) * ldh + i;
                        const float h = *p;
                        *p = acc[a][q] * (1.f - h * h);
                    }
                }
            }
            __syncthreads();
        }
        __syncthreads();
        first = false;
    }
    if (GRAD) {
        // loss partial of this CTA (lane 0 of each warp holds a share)
        __shared__ double lred[kMlpThreads / 32];
        if (lane == 0) lred[warp] = lsum;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < kMlpThreads / 32; ++w) t += lred[w];
            lpart[blockIdx.x] = t;
        }
        // a CTA without tiles contributes zeros
        if (first)
            for (int64_t p = tid; p < D.np; p += kMlpThreads) gmine[p] = 0.f;
    }
    (void)red;
}

// ---------------------------------------------------------------------------
// Tensor-core forward pass (tcgen05) for networks whose hidden layers are all
// 128 wide: 128 samples per tile (one per TMEM lane), 256 threads (warps w
// and w + 4 read the same 32 TMEM lanes and split the 128 columns).  The
// 128 x 128 hidden layers run as BF16 x BF16 -> FP32 MMAs: the activations of
// the tile (A, 128 samples x 128 features) and W_l (B, 128 outputs x 128
// inputs) sit in shared memory in the canonical K-major layout without
// swizzle -- 8 x 8 BF16 core matrices of 128 contiguous bytes, the next core
// matrix along K 128 bytes on, along the rows 16 core matrices on -- and the
// product lands in tensor memory; each thread reads back half a row, adds
// the bias, applies tanh and writes the next layer's BF16 operand.  The first
// layer (input width <= 32) and the scalar output layer run on the FP32 pipe.
// One thread issues the MMAs; their completion is awaited on an mbarrier
// with a bounded wait (on expiry the kernel writes NaN outputs).
// ---------------------------------------------------------------------------
constexpr int kTcM = 128;        // samples per tile = TMEM lanes
constexpr int kTcW = 128;        // hidden width of the tensor-core path

__device__ inline unsigned tc_su32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) of a 128-column K-major operand
__device__ inline int tc_off(int r, int k) { return ((r >> 3) * (kTcW / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2; }

__device__ inline uint64_t tc_desc(const void *base) {
    uint64_t d = (uint64_t)((tc_su32(base) >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;                 // leading byte offset: next core matrix along K
    d |= (uint64_t)((kTcW / 8 * 128) >> 4) << 32;    // stride byte offset: next 8 rows
    d |= (uint64_t)1 << 46;                          // descriptor version
    return d;                                        // base offset 0, no swizzle
}

__device__ inline bool tc_wait(uint64_t *mbar, unsigned parity) {
    for (long it = 0; it < (1l << 26); ++it) {
        unsigned d;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(d) : "r"(tc_su32(mbar)), "r"(parity) : "memory");
        if (d) return true;
    }
    return false;
}

// tanh(x) = 1 - 2 / (1 + e^{2x}) with e^{2x} = 2^{xk}, xk = (2 / ln 2) x, by the
// SFU's base-2 exponential and its reciprocal: absolute error about 1e-7, +-1
// for large |x|; the tensor-core paths round the result to BF16 (8
// significant bits).  The kernels keep the biases and the first layer's
// weights scaled by kTanhK, so that a pre-activation v + b enters as
// fma(v, kTanhK, b kTanhK).
constexpr float kTanhK = 2.88539008f;
__device__ __forceinline__ float tanh_sfu_k(float xk) {
    float e, r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(xk));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.f + e));
    return fmaf(-2.f, r, 1.f);
}

// 8 consecutive floats of shared memory (16-byte aligned)
__device__ __forceinline__ void lds8(const float *p, float (&v)[8]) {
    const float4 a = reinterpret_cast<const float4 *>(p)[0], b = reinterpret_cast<const float4 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// first-layer weights in shared memory with the row stride padded to 4 floats
__host__ __device__ inline int w1_ld(int w0) { return (w0 + 3) & ~3; }

// pre-activation of first-layer output o: b + W_1[o, :] x with 16-byte loads
__device__ __forceinline__ float layer1_dot(const float *sW1, int ld, int w0, int o, float b, const float (&x)[kMlpMaxIn]) {
    float t = b;
    const float4 *w = reinterpret_cast<const float4 *>(sW1 + o * ld);
#pragma unroll
    for (int q = 0; q < kMlpMaxIn / 4; ++q) {
        if (4 * q < w0) {
            const float4 v = w[q];
            t = fmaf(v.x, x[4 * q], t);
            t = fmaf(v.y, x[4 * q + 1], t);
            t = fmaf(v.z, x[4 * q + 2], t);
            t = fmaf(v.w, x[4 * q + 3], t);
        }
    }
    return t;
}

constexpr int kTgMaxMma = 3;
constexpr int kTgN1 = 32;        // first-layer product columns: inputs, a ones row, zero padding
constexpr int kTgTile = kTcM * kTcW * 2;   // bytes of one 128 x 128 BF16 operand

__device__ inline uint64_t tc_desc_mn(const void *base) {
    uint64_t d = (uint64_t)((tc_su32(base) >> 4) & 0x3FFF);
    d |= (uint64_t)((kTcW / 8 * 128) >> 4) << 16;   // leading byte offset: next 8 along K (the stored rows)
    d |= (uint64_t)(128 >> 4) << 32;                 // stride byte offset: next 8 along M / N (the stored columns)
    d |= (uint64_t)1 << 46;
    return d;
}

// kind::f16 instruction descriptor with N columns; a_mn / b_mn select MN-major operands
__host__ __device__ constexpr uint32_t tc_idesc(int n, int a_mn, int b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

__device__ inline void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

__device__ inline void tc_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(tc_su32(mbar)) : "memory");
}

// operands written through the generic proxy become visible to the MMAs, and
// every earlier TMEM read of the CTA is ordered before them
__device__ inline void tc_sync_for_mma() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// bounded wait for the round's commit, the same decision in every thread; on
// expiry a second bounded wait for MMAs still in flight
__device__ inline bool tc_round_wait(uint64_t *mbar, unsigned &parity) {
    const bool got = __syncthreads_and(tc_wait(mbar, parity));
    if (!got) {
        tc_wait(mbar, parity);
        return false;
    }
    parity ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return true;
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes
__device__ inline void tc_ld32(uint32_t addr, float (&v)[32]) {
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

// v[j] summed over the warp's 32 lanes for every j; lane j returns column j
// (five halving exchanges: at each the lanes keep one half and add the
// partner's copy of it)
__device__ inline float warp_transpose_sum(float (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) {
        const bool up = (lane & k) != 0;
#pragma unroll
        for (int j = 0; j < k; ++j) {
            const float send = up ? v[j] : v[j + k];
            const float keep = up ? v[j + k] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, k);
        }
    }
    return v[0];
}

__device__ inline void bf16x8_load(const unsigned char *p, float (&h)[8]) {
    const uint4 u = *reinterpret_cast<const uint4 *>(p);
    const __nv_bfloat162 *b = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 f = __bfloat1622float2(b[j]);
        h[2 * j] = f.x;
        h[2 * j + 1] = f.y;
    }
}

__device__ inline void bf16x8_store(unsigned char *p, const float (&h)[8]) {
    __align__(16) __nv_bfloat162 b[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = __floats2bfloat162_rn(h[2 * j], h[2 * j + 1]);
    *reinterpret_cast<uint4 *>(p) = *reinterpret_cast<const uint4 *>(b);
}

// P threads per sample (128 P per CTA), each with 128 / P columns of its row
template <int P>
__global__ void __launch_bounds__(128 * P, 1) k_mlp_fwd_tc(MlpDesc D, const float *__restrict__ theta,
                                                           const float *__restrict__ X, int64_t n,
                                                           float *__restrict__ Y) {
    constexpr int NT = 128 * P, CW = 128 / P;
    extern __shared__ __align__(1024) unsigned char tsm[];
    const int L = D.L, n_mma = L - 2, w0 = D.w[0];
    unsigned char *sWm = tsm;                                  // n_mma x 32 KB: W_2 .. W_{L-1} (BF16)
    unsigned char *sAct = sWm + (size_t)n_mma * kTgTile;       // 2 x 32 KB: activations (BF16)
    float *sW1 = reinterpret_cast<float *>(sAct + 2 * kTgTile);   // kTcW x w1_ld(w0)
    float *sB = sW1 + kTcW * w1_ld(w0);                        // biases of layers 1 .. L-1 (kTcW each)
    float *sWL = sB + (L - 1) * kTcW;                          // output weights (kTcW) and bias
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ float sY[P][kTcM];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = 32 * (warp & 3) + lane, cb = CW * (warp >> 2);
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    // weights once per CTA
    for (int l = 2; l < L; ++l) {
        const float *W = theta + D.off[l];
        unsigned char *dst = sWm + (size_t)(l - 2) * kTgTile;
        for (int e = tid; e < kTcW * kTcW; e += NT) {
            const int o = e / kTcW, i = e % kTcW;
            *reinterpret_cast<__nv_bfloat16 *>(dst + tc_off(o, i)) = __float2bfloat16_rn(__ldg(W + e));
        }
    }
    for (int e = tid; e < kTcW * w1_ld(w0); e += NT) {
        const int o = e / w1_ld(w0), i = e % w1_ld(w0);
        sW1[e] = i < w0 ? kTanhK * __ldg(theta + D.off[1] + o * w0 + i) : 0.f;
    }
    for (int l = 1; l < L; ++l)
        for (int o = tid; o < kTcW; o += NT)
            sB[(l - 1) * kTcW + o] = kTanhK * __ldg(theta + D.off[l] + (int64_t)kTcW * D.w[l - 1] + o);
    for (int i = tid; i <= kTcW; i += NT) sWL[i] = __ldg(theta + D.off[L] + i);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_su32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_su32(&tmem_base)), "r"(kTcW) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    unsigned parity = 0;
    bool ok = true;
    const int64_t n_tiles = (n + kTcM - 1) / kTcM;
    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        const int64_t s = tile * kTcM + row;   // this thread's sample
        // layer 1 on the FP32 pipe: h_1 = tanh(W_1 x + b_1) over this thread's 64 columns
        {
            float x[kMlpMaxIn];
#pragma unroll
            for (int i = 0; i < kMlpMaxIn; ++i) x[i] = (i < w0 && s < n) ? __ldg(X + s * w0 + i) : 0.f;
            for (int o0 = cb; o0 < cb + CW; o0 += 8) {
                float hv[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int o = o0 + j;
                    hv[j] = tanh_sfu_k(layer1_dot(sW1, w1_ld(w0), w0, o, sB[o], x));
                }
                bf16x8_store(sAct + tc_off(row, o0), hv);
            }
        }
        float yv = 0.f;
        for (int l = 2; l < L; ++l) {
            const unsigned char *Ain = sAct + (size_t)((l - 2) & 1) * kTgTile;
            unsigned char *Aout = sAct + (size_t)((l - 1) & 1) * kTgTile;
            tc_sync_for_mma();
            if (tid == 0) {
                const unsigned char *Bw = sWm + (size_t)(l - 2) * kTgTile;
                for (int kk = 0; kk < kTcW / 16; ++kk)
                    tc_mma(tmem, tc_desc(Ain + kk * 256), tc_desc(Bw + kk * 256), tc_idesc(kTcW, 0, 0), kk > 0);
                tc_commit(&mbar);
            }
            if (!tc_round_wait(&mbar, parity)) {
                ok = false;
                break;
            }
            const float *bl = sB + (l - 1) * kTcW;
            const bool last = l == L - 1;
            for (int c0 = cb; c0 < cb + CW; c0 += 32) {
                float v[32];
                tc_ld32(tmem + lane_off + (uint32_t)c0, v);
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    float hv[8], bk[8];
                    lds8(bl + c0 + 8 * g, bk);
#pragma unroll
                    for (int j = 0; j < 8; ++j) hv[j] = tanh_sfu_k(fmaf(v[8 * g + j], kTanhK, bk[j]));
                    if (last) {
                        float wl[8];
                        lds8(sWL + c0 + 8 * g, wl);
#pragma unroll
                        for (int j = 0; j < 8; ++j) yv = fmaf(hv[j], wl[j], yv);
                    } else {
                        bf16x8_store(Aout + tc_off(row, c0 + 8 * g), hv);
                    }
                }
            }
        }
        if (!ok) break;
        sY[warp >> 2][row] = yv;
        __syncthreads();
        if (warp < 4 && s < n) {
            float t = sY[0][row];
#pragma unroll
            for (int q = 1; q < P; ++q) t += sY[q][row];
            Y[s] = t + sWL[kTcW];
        }
    }
    if (!ok) {
        for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
            const int64_t s = tile * kTcM + row;
            if (warp < 4 && s < n) Y[s] = __int_as_float(0x7fc00000);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcW) : "memory");
}

static bool mlp_tc_shape(const MlpDesc &D) {
    if (D.L < 3) return false;
    for (int l = 1; l < D.L; ++l)
        if (D.w[l] != kTcW) return false;
    return D.w[0] <= kMlpMaxIn;
}

static size_t mlp_tc_smem(const MlpDesc &D) {
    return (size_t)(D.L - 2) * kTcW * kTcW * 2 + 2 * (size_t)kTcM * kTcW * 2 +
           4 * ((size_t)kTcW * w1_ld(D.w[0]) + (size_t)(D.L - 1) * kTcW + kTcW + 1) + 64;
}

// ---------------------------------------------------------------------------
// Tensor-core loss gradient (tcgen05) for networks whose hidden layers are
// all 128 wide, with one to three 128 x 128 layers (L = 3 .. 5).  128
// samples per tile, 256 threads: the two threads of a sample (warps w and
// w + 4 share TMEM lanes 32 (w % 4) ..) split the 128 columns of every
// epilogue.  Every operand stays in the layout the forward pass writes --
// activations and errors as (sample, feature) and W_l as (output, input),
// K-major without swizzle -- and the backward pass reads the transposes it
// needs through MN-major descriptors (the same bytes with the two strides
// swapped).  Per tile:
//   forward   layer 1 on the FP32 pipe, the hidden layers as BF16 MMAs into
//             a 128-column TMEM working region, the scalar output in FP32;
//   output    e = 2 (y - t) / n; dW_L and db_L; e_{L-1} = e w_L (1 - h^2);
//   layer l   one round of two MMAs: working = e_l W_l (propagation) and
//             dW_l += e_l^T h_{l-1} (a 128-column TMEM accumulator that
//             persists over the CTA's tiles); e_{l-1} = working (1 - h^2);
//   layer 1   dW_1 and db_1 = e_1^T [x, 1] by one N = 32 MMA, summed over
//             tiles in registers (thread = output row).
// Bias gradients of the hidden layers and dW_L are column sums over the
// tile's samples, formed by transposing warp sums in the epilogues.  h_1 is
// recomputed in the backward pass, so max(2, L - 2) activation buffers of
// 32 KB suffice.  The product of 1 - h^2 uses h as the BF16 operand holds
// it.  Waits are bounded; on expiry the CTA's gradient slice is NaN.
// ---------------------------------------------------------------------------
struct TgLayout {
    int nm, nb;
    size_t w, buf, x, w1, b, wl, acc, total;
};

__host__ __device__ inline TgLayout tg_layout(const MlpDesc &D) {
    TgLayout t;
    t.nm = D.L - 2;
    t.nb = t.nm > 2 ? t.nm : 2;
    t.w = 0;
    t.buf = t.w + (size_t)t.nm * kTgTile;
    t.x = t.buf + (size_t)t.nb * kTgTile;
    t.w1 = t.x + (size_t)kTgN1 * kTcM * 2;
    t.b = t.w1 + (size_t)kTcW * w1_ld(D.w[0]) * 4;
    t.wl = t.b + (size_t)(D.L - 1) * kTcW * 4;
    t.acc = t.wl + 132 * 4;
    t.total = t.acc + (size_t)4 * (t.nm + 1) * kTcW * 4;
    return t;
}

template <int P>
__global__ void __launch_bounds__(128 * P, 1)
    k_mlp_grad_tc(MlpDesc D, const float *__restrict__ theta, const float *__restrict__ X,
                  const float *__restrict__ T, int64_t n, float *__restrict__ gpart, double *__restrict__ lpart,
                  float inv_n) {
    constexpr int NT = 128 * P, CW = 128 / P, NG = kTgN1 / P;
    extern __shared__ __align__(1024) unsigned char tsm[];
    const TgLayout Ly = tg_layout(D);
    const int L = D.L, nm = Ly.nm, w0 = D.w[0];
    unsigned char *sW = tsm + Ly.w;                                  // W_2 .. W_{L-1}, BF16 (output, input)
    unsigned char *sBuf = tsm + Ly.buf;                              // activation / error buffers
    unsigned char *sX = tsm + Ly.x;                                  // [x, 1, 0] as (input, sample), BF16
    float *sW1 = reinterpret_cast<float *>(tsm + Ly.w1);             // W_1, FP32 (output, input), padded rows
    float *sB = reinterpret_cast<float *>(tsm + Ly.b);               // b_1 .. b_{L-1}
    float *sWL = reinterpret_cast<float *>(tsm + Ly.wl);             // w_L and b_L
    float *sAcc = reinterpret_cast<float *>(tsm + Ly.acc);           // per lane group: db_2 .. db_{L-1}, dW_L
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ float sY[P][kTcM];
    __shared__ double sL[NT / 32];
    __shared__ float sE[NT / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = 32 * (warp & 3) + lane;       // sample of the tile (and TMEM lane)
    const int part = warp >> 2;                   // columns CW part .. CW part + CW - 1
    const int cb = CW * part;
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    auto buf = [&](int i) { return sBuf + (size_t)i * kTgTile; };
    // buffer of h_l: h_1 and h_{L-1} in buffer 0, h_l (2 <= l <= L-2) in buffer l-1;
    // h_1 is recomputed for the backward pass into buffer 0 (L > 3) or 1 (L = 3)
    auto hbuf = [&](int l) { return (l == 1 || l == L - 1) ? buf(0) : buf(l - 1); };
    unsigned char *sR = nm >= 2 ? buf(0) : buf(1);

    for (int l = 2; l < L; ++l) {
        const float *W = theta + D.off[l];
        unsigned char *dst = sW + (size_t)(l - 2) * kTgTile;
        for (int e = tid; e < kTcW * kTcW; e += NT) {
            const int o = e / kTcW, i = e % kTcW;
            *reinterpret_cast<__nv_bfloat16 *>(dst + tc_off(o, i)) = __float2bfloat16_rn(__ldg(W + e));
        }
    }
    for (int e = tid; e < kTcW * w1_ld(w0); e += NT) {
        const int o = e / w1_ld(w0), i = e % w1_ld(w0);
        sW1[e] = i < w0 ? kTanhK * __ldg(theta + D.off[1] + o * w0 + i) : 0.f;
    }
    for (int l = 1; l < L; ++l)
        for (int o = tid; o < kTcW; o += NT)
            sB[(l - 1) * kTcW + o] = kTanhK * __ldg(theta + D.off[l] + (int64_t)kTcW * D.w[l - 1] + o);
    for (int i = tid; i <= kTcW; i += NT) sWL[i] = __ldg(theta + D.off[L] + i);
    for (int e = tid; e < 4 * (nm + 1) * kTcW; e += NT) sAcc[e] = 0.f;
    for (int e = tid; e < kTgN1 * kTcM / 8; e += NT) reinterpret_cast<uint4 *>(sX)[e] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_su32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_su32(&tmem_base)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t twork = tmem + lane_off;
    unsigned parity = 0;
    bool ok = true, first = true;
    double lsum = 0.0;
    float gb_out = 0.f;            // db_L share of this thread (part 0 only)
    float gW1[NG];                 // dW_1 row `row`, columns NG part .. NG part + NG - 1 of [x, 1, 0]
#pragma unroll
    for (int j = 0; j < NG; ++j) gW1[j] = 0.f;
    float xr[kMlpMaxIn];

    // h_1 of this thread's sample over its 64 columns, rounded to BF16 into dst
    auto layer1 = [&](unsigned char *dst) {
        for (int o0 = cb; o0 < cb + CW; o0 += 8) {
            float hv[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int o = o0 + j;
                hv[j] = tanh_sfu_k(layer1_dot(sW1, w1_ld(w0), w0, o, sB[o], xr));
            }
            bf16x8_store(dst + tc_off(row, o0), hv);
        }
    };

    const int64_t n_tiles = (n + kTcM - 1) / kTcM;
    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        const int64_t s = tile * kTcM + row;
        const bool valid = s < n;
#pragma unroll
        for (int i = 0; i < kMlpMaxIn; ++i) xr[i] = (i < w0 && valid) ? __ldg(X + s * w0 + i) : 0.f;
        // [x, 1] of the sample as column `row` of the first-layer operand (part 0 writes it)
        if (part == 0) {
#pragma unroll
            for (int i = 0; i < kMlpMaxIn; ++i)
                if (i <= w0)
                    *reinterpret_cast<__nv_bfloat16 *>(sX + tc_off(i, row)) =
                        __float2bfloat16_rn(i < w0 ? xr[i] : (valid ? 1.f : 0.f));
        }
        layer1(buf(0));
        // ---- forward through the hidden 128 x 128 layers
        float yp = 0.f;
        for (int l = 2; l < L && ok; ++l) {
            tc_sync_for_mma();
            if (tid == 0) {
                const unsigned char *A = hbuf(l - 1), *Bw = sW + (size_t)(l - 2) * kTgTile;
                for (int kk = 0; kk < kTcW / 16; ++kk)
                    tc_mma(tmem, tc_desc(A + kk * 256), tc_desc(Bw + kk * 256), tc_idesc(kTcW, 0, 0), kk > 0);
                tc_commit(&mbar);
            }
            if (!tc_round_wait(&mbar, parity)) {
                ok = false;
                break;
            }
            const float *bl = sB + (l - 1) * kTcW;
            unsigned char *out = hbuf(l);
            const bool last = l == L - 1;
            for (int c0 = cb; c0 < cb + CW; c0 += 32) {
                float v[32];
                tc_ld32(twork + (uint32_t)c0, v);
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    float hv[8], bk[8];
                    lds8(bl + c0 + 8 * g, bk);
#pragma unroll
                    for (int j = 0; j < 8; ++j) hv[j] = tanh_sfu_k(fmaf(v[8 * g + j], kTanhK, bk[j]));
                    if (last) {
                        float wl[8];
                        lds8(sWL + c0 + 8 * g, wl);
#pragma unroll
                        for (int j = 0; j < 8; ++j) yp = fmaf(hv[j], wl[j], yp);
                    }
                    bf16x8_store(out + tc_off(row, c0 + 8 * g), hv);
                }
            }
        }
        if (!ok) break;
        // ---- output layer: y, e = 2 (y - t) / n, dW_L, db_L, e_{L-1}
        sY[part][row] = yp;
        __syncthreads();
        float ysum = sY[0][row];
#pragma unroll
        for (int q = 1; q < P; ++q) ysum += sY[q][row];
        const float y = ysum + sWL[kTcW];
        const float dlt = valid ? y - __ldg(T + s) : 0.f;
        if (part == 0) {
            lsum += (double)dlt * (double)dlt;
            gb_out += 2.f * dlt * inv_n;
        }
        const float ey = 2.f * dlt * inv_n;
        {
            unsigned char *H = hbuf(L - 1);
            for (int c0 = cb; c0 < cb + CW; c0 += 32) {
                float d[32], g[32];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float hb[8], wl[8];
                    bf16x8_load(H + tc_off(row, c0 + 8 * q), hb);
                    lds8(sWL + c0 + 8 * q, wl);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        g[8 * q + j] = ey * hb[j];
                        d[8 * q + j] = ey * wl[j] * (1.f - hb[j] * hb[j]);
                    }
                    float dq[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) dq[j] = d[8 * q + j];
                    bf16x8_store(H + tc_off(row, c0 + 8 * q), dq);
                }
                const float sg = warp_transpose_sum(g);
                sAcc[((warp & 3) * (nm + 1) + nm) * kTcW + c0 + lane] += sg;
                const float sd = warp_transpose_sum(d);
                sAcc[((warp & 3) * (nm + 1) + (L - 1 - 2)) * kTcW + c0 + lane] += sd;
            }
        }
        // ---- backward through the hidden layers: e_l W_l and dW_l += e_l^T h_{l-1}
        for (int l = L - 1; l >= 2 && ok; --l) {
            if (l == 2) layer1(sR);
            unsigned char *E = hbuf(l);
            unsigned char *H = l - 1 == 1 ? sR : hbuf(l - 1);
            tc_sync_for_mma();
            if (tid == 0) {
                const unsigned char *Bw = sW + (size_t)(l - 2) * kTgTile;
                const uint32_t tacc = tmem + (uint32_t)(kTcW * (l - 1));
                for (int kk = 0; kk < kTcW / 16; ++kk)
                    tc_mma(tmem, tc_desc(E + kk * 256), tc_desc_mn(Bw + kk * 4096), tc_idesc(kTcW, 0, 1), kk > 0);
                for (int kk = 0; kk < kTcM / 16; ++kk)
                    tc_mma(tacc, tc_desc_mn(E + kk * 4096), tc_desc_mn(H + kk * 4096), tc_idesc(kTcW, 1, 1),
                           (kk > 0 || !first) ? 1u : 0u);
                tc_commit(&mbar);
            }
            if (!tc_round_wait(&mbar, parity)) {
                ok = false;
                break;
            }
            for (int c0 = cb; c0 < cb + CW; c0 += 32) {
                float d[32];
                tc_ld32(twork + (uint32_t)c0, d);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float hb[8], dq[8];
                    bf16x8_load(H + tc_off(row, c0 + 8 * q), hb);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        d[8 * q + j] *= 1.f - hb[j] * hb[j];
                        dq[j] = d[8 * q + j];
                    }
                    bf16x8_store(H + tc_off(row, c0 + 8 * q), dq);
                }
                if (l - 1 >= 2) {
                    const float sd = warp_transpose_sum(d);
                    sAcc[((warp & 3) * (nm + 1) + (l - 1 - 2)) * kTcW + c0 + lane] += sd;
                }
            }
        }
        if (!ok) break;
        // ---- dW_1 and db_1 = e_1^T [x, 1]
        tc_sync_for_mma();
        if (tid == 0) {
            for (int kk = 0; kk < kTcM / 16; ++kk)
                tc_mma(tmem, tc_desc_mn(sR + kk * 4096), tc_desc(sX + kk * 256), tc_idesc(kTgN1, 1, 0), kk > 0);
            tc_commit(&mbar);
        }
        if (!tc_round_wait(&mbar, parity)) {
            ok = false;
            break;
        }
        {
            float v[32];
            tc_ld32(twork, v);
#pragma unroll
            for (int j = 0; j < NG; ++j) {
#pragma unroll
                for (int q = 0; q < P; ++q)
                    if (q == part) gW1[j] += v[NG * q + j];
            }
        }
        first = false;
    }

    // ---- the CTA's gradient slice
    float *g = gpart + (int64_t)blockIdx.x * D.np;
    tc_sync_for_mma();
    if (ok) {
        for (int l = 2; l < L; ++l) {
            const uint32_t tacc = tmem + (uint32_t)(kTcW * (l - 1)) + lane_off;
            for (int c0 = cb; c0 < cb + CW; c0 += 32) {
                float v[32];
                tc_ld32(tacc + (uint32_t)c0, v);
                float *p = g + D.off[l] + (int64_t)row * kTcW + c0;
#pragma unroll
                for (int j = 0; j < 32; ++j) p[j] = first ? 0.f : v[j];
            }
        }
        for (int o = tid; o < kTcW; o += NT) {
            for (int v = 0; v <= nm; ++v) {
                float t = 0.f;
                for (int w = 0; w < 4; ++w) t += sAcc[(w * (nm + 1) + v) * kTcW + o];
                if (v < nm) g[D.off[v + 2] + (int64_t)kTcW * kTcW + o] = t;
                else g[D.off[L] + o] = t;
            }
        }
#pragma unroll
        for (int j = 0; j < NG; ++j) {
            const int i = NG * part + j;
            if (i < w0) g[D.off[1] + (int64_t)row * w0 + i] = gW1[j];
            else if (i == w0) g[D.off[1] + (int64_t)kTcW * w0 + row] = gW1[j];
        }
    }
    float t = gb_out;
    double ls = lsum;
    for (int o = 16; o; o >>= 1) {
        t += __shfl_xor_sync(0xffffffffu, t, o);
        ls += __shfl_xor_sync(0xffffffffu, ls, o);
    }
    if (lane == 0) {
        sE[warp] = t;
        sL[warp] = ls;
    }
    __syncthreads();
    if (tid == 0) {
        float te = 0.f;
        double tl = 0.0;
        for (int w = 0; w < NT / 32; ++w) {
            te += sE[w];
            tl += sL[w];
        }
        if (ok) g[D.off[L] + kTcW] = te;
        lpart[blockIdx.x] = ok ? tl : (double)__int_as_float(0x7fc00000);
    }
    if (!ok)
        for (int64_t p = tid; p < D.np; p += NT) g[p] = __int_as_float(0x7fc00000);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

static bool mlp_tg_shape(const MlpDesc &D) {
    return mlp_tc_shape(D) && D.L - 2 <= kTgMaxMma && D.w[0] < kTgN1 && tg_layout(D).total <= 224 * 1024;
}

static int g_mlp_tc = 1;
void set_mlp_tensor_cores(int on) { g_mlp_tc = on; }
// threads per sample of the tensor-core kernels: 2 (256 per CTA) or 4 (512)
static int g_mlp_tc_parts = 4;
void set_mlp_tc_threads(int threads) { g_mlp_tc_parts = threads / 128; }

// grad[p] = sum over CTA slices (fixed order); loss = sum of partials / n.
__global__ void k_mlp_reduce(const float *__restrict__ gpart, int nslices, int64_t np, float *__restrict__ grad,
                             const double *__restrict__ lpart, float *__restrict__ loss, double inv_n) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        float t = 0.f;
        for (int c = 0; c < nslices; ++c) t += gpart[(int64_t)c * np + p];
        grad[p] = t;
    }
    if (loss && blockIdx.x == 0 && threadIdx.x == 0) {
        double t = 0.0;
        for (int c = 0; c < nslices; ++c) t += lpart[c];
        *loss = (float)(t * inv_n);
    }
}

// Adam (Kingma and Ba 2015) with bias corrections c1 = 1 - b1^t, c2 = 1 - b2^t.
__global__ void k_adam(int64_t n, float *__restrict__ theta, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

static int mlp_grid(int64_t n) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (n + kTS - 1) / kTS;
    int64_t g = tiles < nsm ? tiles : nsm;
    if (g > kMlpMaxCtas) g = kMlpMaxCtas;
    return (int)(g < 1 ? 1 : g);
}

rfm_status mlp_nparams(const rfm_mlp *net, int64_t *np) {
    MlpDesc D;
    rfm_status rc = mlp_desc(net, &D);
    if (rc == RFM_OK) *np = D.np;
    return rc;
}

size_t mlp_workspace_bytes(const MlpDesc &D) {
    return ((size_t)kMlpMaxCtas * D.np * 4 + 255) / 256 * 256 + (size_t)kMlpMaxCtas * 8;
}

rfm_status mlp_workspace(const rfm_mlp *net, size_t *bytes) {
    MlpDesc D;
    rfm_status rc = mlp_desc(net, &D);
    if (rc == RFM_OK) *bytes = mlp_workspace_bytes(D);
    return rc;
}

rfm_status launch_mlp_forward(const rfm_mlp *net, const float *theta, const float *X, int64_t n, float *Y,
                              cudaStream_t st) {
    MlpDesc D;
    rfm_status rc = mlp_desc(net, &D);
    if (rc != RFM_OK) return rc;
    if (n <= 0) return RFM_OK;
    if (g_mlp_tc && mlp_tc_shape(D) && mlp_tc_smem(D) <= 200 * 1024) {
        const size_t smem = mlp_tc_smem(D);
        RFM_CUDA_CHECK(cudaFuncSetAttribute(k_mlp_fwd_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        RFM_CUDA_CHECK(cudaFuncSetAttribute(k_mlp_fwd_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int dev = 0, nsm = 0;
        RFM_CUDA_CHECK(cudaGetDevice(&dev));
        RFM_CUDA_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        const int64_t tiles = (n + kTcM - 1) / kTcM;
        const int grid = (int)(tiles < nsm ? tiles : nsm);
        ProfScope ps("k_mlp_fwd_tc", st);
        if (g_mlp_tc_parts == 4) k_mlp_fwd_tc<4><<<grid, 512, smem, st>>>(D, theta, X, n, Y);
        else k_mlp_fwd_tc<2><<<grid, 256, smem, st>>>(D, theta, X, n, Y);
        RFM_CUDA_CHECK(cudaGetLastError());
        return RFM_OK;
    }
    const size_t smem = (size_t)D.smem_floats * 4;
    RFM_CUDA_CHECK(cudaFuncSetAttribute(k_mlp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, nsm = 0;
    RFM_CUDA_CHECK(cudaGetDevice(&dev));
    RFM_CUDA_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int64_t tiles = (n + kTS - 1) / kTS;
    const int grid = (int)(tiles < 4 * (int64_t)nsm ? tiles : 4 * (int64_t)nsm);
    ProfScope ps("k_mlp_forward", st);
    k_mlp<false><<<grid, kMlpThreads, smem, st>>>(D, theta, X, nullptr, n, Y, nullptr, nullptr, 0.f);
    RFM_CUDA_CHECK(cudaGetLastError());
    return RFM_OK;
}

rfm_status launch_mlp_grad(const rfm_mlp *net, const float *theta, const float *X, const float *T, int64_t n,
                           float *grad, float *loss, void *ws, size_t ws_bytes, cudaStream_t st) {
    MlpDesc D;
    rfm_status rc = mlp_desc(net, &D);
    if (rc != RFM_OK) return rc;
    if (n <= 0) {
        set_error("rfm_mlp_grad: empty batch");
        return RFM_EINVAL;
    }
    if (!ws || ws_bytes < mlp_workspace_bytes(D) || ((uintptr_t)ws & 255)) {
        set_error("rfm_mlp_grad: workspace must be 256-byte aligned with at least %zu bytes", mlp_workspace_bytes(D));
        return RFM_ENOSPACE;
    }
    float *gpart = ws_ptr<float>(ws, 0);
    double *lpart = ws_ptr<double>(ws, ((size_t)kMlpMaxCtas * D.np * 4 + 255) / 256 * 256);
    int grid;
    if (g_mlp_tc && mlp_tg_shape(D)) {
        const size_t smem = tg_layout(D).total;
        RFM_CUDA_CHECK(cudaFuncSetAttribute(k_mlp_grad_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        RFM_CUDA_CHECK(cudaFuncSetAttribute(k_mlp_grad_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int dev = 0, nsm = 0;
        RFM_CUDA_CHECK(cudaGetDevice(&dev));
        RFM_CUDA_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        const int64_t tiles = (n + kTcM - 1) / kTcM;
        grid = (int)(tiles < nsm ? tiles : nsm);
        if (grid > kMlpMaxCtas) grid = kMlpMaxCtas;
        ProfScope ps("k_mlp_grad_tc", st);
        if (g_mlp_tc_parts == 4)
            k_mlp_grad_tc<4><<<grid, 512, smem, st>>>(D, theta, X, T, n, gpart, lpart, (float)(1.0 / n));
        else
            k_mlp_grad_tc<2><<<grid, 256, smem, st>>>(D, theta, X, T, n, gpart, lpart, (float)(1.0 / n));
        RFM_CUDA_CHECK(cudaGetLastError());
    } else {
        const size_t smem = (size_t)D.smem_floats * 4;
        RFM_CUDA_CHECK(cudaFuncSetAttribute(k_mlp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        grid = mlp_grid(n);
        ProfScope ps("k_mlp_grad", st);
        k_mlp<true><<<grid, kMlpThreads, smem, st>>>(D, theta, X, T, n, nullptr, gpart, lpart, (float)(1.0 / n));
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    {
        ProfScope ps("k_mlp_reduce", st);
        k_mlp_reduce<<<(unsigned)((D.np + 255) / 256), 256, 0, st>>>(gpart, grid, D.np, grad, lpart, loss,
                                                                      1.0 / (double)n);
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    return RFM_OK;
}

// Minibatch gather: xb[s, :] = X[order[s], :], tb[s] = T[order[s]].
__global__ void k_gather_batch(const float *__restrict__ X, const float *__restrict__ T,
                               const int64_t *__restrict__ order, int batch, int w0, float *__restrict__ xb,
                               float *__restrict__ tb) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)batch * (w0 + 1);
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = e / (w0 + 1);
        const int i = (int)(e - s * (w0 + 1));
        const int64_t src = order[s];
        if (i < w0) xb[s * w0 + i] = X[src * w0 + i];
        else tb[s] = T[src];
    }
}

// Workspace of the training loop: the gradient's workspace, the gradient,
// and the gathered batch.
static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

size_t mlp_train_bytes(const MlpDesc &D, int batch) {
    return align256(mlp_workspace_bytes(D)) + align256((size_t)D.np * 4) + align256((size_t)batch * D.w[0] * 4) +
           align256((size_t)batch * 4);
}

rfm_status mlp_train_size(const rfm_mlp *net, int batch, size_t *bytes) {
    MlpDesc D;
    rfm_status rc = mlp_desc(net, &D);
    if (rc != RFM_OK) return rc;
    if (batch < 1) {
        set_error("rfm_mlp_train_size: batch must be >= 1");
        return RFM_EINVAL;
    }
    *bytes = mlp_train_bytes(D, batch);
    return RFM_OK;
}

rfm_status launch_adam(int64_t n, float *theta, float *m, float *v, const float *g, int t, float lr, float b1,
                       float b2, float eps, cudaStream_t st);

rfm_status launch_mlp_train(const rfm_mlp *net, float *theta, float *m, float *v, const float *X, const float *T,
                            const int64_t *order, int batch, int n_steps, int t0, const float *lr, float b1, float b2,
                            float eps, float *loss, void *ws, size_t ws_bytes, cudaStream_t st) {
    MlpDesc D;
    rfm_status rc = mlp_desc(net, &D);
    if (rc != RFM_OK) return rc;
    if (batch < 1 || n_steps < 0 || t0 < 1) {
        set_error("rfm_mlp_train: need batch >= 1, n_steps >= 0, t0 >= 1");
        return RFM_EINVAL;
    }
    const size_t need = mlp_train_bytes(D, batch);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) {
        set_error("rfm_mlp_train: workspace must be 256-byte aligned with at least %zu bytes", need);
        return RFM_ENOSPACE;
    }
    char *w = static_cast<char *>(ws);
    const size_t gws = align256(mlp_workspace_bytes(D));
    float *g = reinterpret_cast<float *>(w + gws);
    float *xb = reinterpret_cast<float *>(w + gws + align256((size_t)D.np * 4));
    float *tb = reinterpret_cast<float *>(w + gws + align256((size_t)D.np * 4) + align256((size_t)batch * D.w[0] * 4));
    const int64_t work = (int64_t)batch * (D.w[0] + 1);
    const unsigned gblocks = (unsigned)((work + 255) / 256 < 1024 ? (work + 255) / 256 : 1024);
    for (int k = 0; k < n_steps; ++k) {
        {
            ProfScope ps("k_gather_batch", st);
            k_gather_batch<<<gblocks, 256, 0, st>>>(X, T, order + (int64_t)k * batch, batch, D.w[0], xb, tb);
            RFM_CUDA_CHECK(cudaGetLastError());
        }
        rc = launch_mlp_grad(net, theta, xb, tb, batch, g, loss ? loss + k : nullptr, ws, gws, st);
        if (rc != RFM_OK) return rc;
        rc = launch_adam(D.np, theta, m, v, g, t0 + k, lr[k], b1, b2, eps, st);
        if (rc != RFM_OK) return rc;
    }
    return RFM_OK;
}

rfm_status launch_adam(int64_t n, float *theta, float *m, float *v, const float *g, int t, float lr, float b1,
                       float b2, float eps, cudaStream_t st) {
    if (n <= 0 || t < 1 || !(lr >= 0.f) || !(b1 >= 0.f && b1 < 1.f) || !(b2 >= 0.f && b2 < 1.f) || !(eps > 0.f)) {
        set_error("rfm_adam_step: need n > 0, t >= 1, lr >= 0, 0 <= b1, b2 < 1, eps > 0");
        return RFM_EINVAL;
    }
    const double c1 = 1.0 - pow((double)b1, (double)t), c2 = 1.0 - pow((double)b2, (double)t);
    ProfScope ps("k_adam", st);
    const int64_t blocks = (n + 255) / 256;
    k_adam<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(n, theta, m, v, g, lr, b1, b2, eps, (float)c1,
                                                                      (float)c2);
    RFM_CUDA_CHECK(cudaGetLastError());
    return RFM_OK;
}

}  // namespace rfm
