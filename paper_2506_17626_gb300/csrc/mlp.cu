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
    const size_t smem = (size_t)D.smem_floats * 4;
    RFM_CUDA_CHECK(cudaFuncSetAttribute(k_mlp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = mlp_grid(n);
    {
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
