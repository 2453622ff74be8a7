// rrqr.cu -- local sigma-RRQR filtering (Algorithm 1) and the operator blocks
// of the right preconditioner (Sec. 3.2, Proposition 3.1).
//
// k_qrcp: one CTA per block, FP64 Householder QR with column pivoting on a
// working copy W of M_j (column-major, leading dimension ldm).  Step k:
//   1. pivot = trailing column of largest norm (norms kept in shared memory,
//      ties to the lowest original index), swapped into place;
//   2. ||W[k:m, k]|| recomputed exactly; stop when it is 0 or < tol |R_11|;
//   3. reflector beta = -sign(alpha) ||x||, v = x / (alpha - beta), v_0 = 1,
//      tau = (beta - alpha) / beta (v stored below the diagonal);
//   4. every trailing column c: s = tau v^T W[k:m, c], W[k:m, c] -= s v
//      (one warp per column), then its norm is downdated,
//      ||W[k+1:m, c]||^2 = ||W[k:m, c]||^2 - W[k, c]^2, and recomputed
//      exactly when cancellation has eaten more than half the digits since
//      the last exact value (the downdated value's relative error grows like
//      eps (norm at last recompute / current norm)^2).
// FP64 throughput is the bound: per element of the trailing matrix one FMA
// for the dot product and one for the update.
#include "device.cuh"
#include "prof.cuh"

namespace rfm {

struct ArgMax {
    double v;
    int p, c;
};

__device__ inline bool better(double v1, int p1, double v2, int p2) { return v1 > v2 || (v1 == v2 && p1 < p2); }

template <typename TM>
__global__ void __launch_bounds__(256) k_qrcp(const BlkRec *__restrict__ blks, const TM *__restrict__ M,
                                              double *__restrict__ W, double *__restrict__ tau,
                                              int32_t *__restrict__ perm_out, int32_t *__restrict__ rank_out,
                                              double *__restrict__ r11_out, double tol) {
    extern __shared__ double smem[];
    const BlkRec B = blks[blockIdx.x];
    const int m = B.m, K = B.K, ld = B.ldm;
    double *cn = smem;             // K current trailing norms
    double *cn0 = smem + K;        // K norms at the last exact recompute
    int *perm = (int *)(smem + 2 * K);
    __shared__ double red_v[8];
    __shared__ int red_p[8], red_c[8];
    __shared__ double s_nx;
    __shared__ int s_piv;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double *Wb = W + B.moff;
    const TM *Mb = M + B.moff;

    // working copy in FP64
    for (int c = warp; c < K; c += 8)
        for (int i = lane; i < m; i += 32) Wb[(int64_t)c * ld + i] = (double)Mb[(int64_t)c * ld + i];
    __syncthreads();
    for (int c = warp; c < K; c += 8) {
        double s = 0.0;
        for (int i = lane; i < m; i += 32) {
            double a = Wb[(int64_t)c * ld + i];
            s = fma(a, a, s);
        }
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            cn[c] = sqrt(s);
            cn0[c] = cn[c];
            perm[c] = c;
        }
    }
    __syncthreads();

    const int steps = m < K ? m : K;
    const double tol3z = sqrt(2.220446049250313e-16);
    double R11 = 0.0;
    int rank = steps;
    for (int k = 0; k < steps; ++k) {
        // 1. pivot
        double bv = -1.0;
        int bp = 0x7fffffff, bc = k;
        for (int c = k + tid; c < K; c += 256)
            if (better(cn[c], perm[c], bv, bp)) { bv = cn[c]; bp = perm[c]; bc = c; }
        for (int o = 16; o; o >>= 1) {
            double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
            int p2 = __shfl_xor_sync(0xffffffffu, bp, o);
            int c2 = __shfl_xor_sync(0xffffffffu, bc, o);
            if (better(v2, p2, bv, bp)) { bv = v2; bp = p2; bc = c2; }
        }
        if (lane == 0) { red_v[warp] = bv; red_p[warp] = bp; red_c[warp] = bc; }
        __syncthreads();
        if (tid == 0) {
            double v = red_v[0];
            int p = red_p[0], c = red_c[0];
            for (int w = 1; w < 8; ++w)
                if (better(red_v[w], red_p[w], v, p)) { v = red_v[w]; p = red_p[w]; c = red_c[w]; }
            s_piv = c;
        }
        __syncthreads();
        const int piv = s_piv;
        if (piv != k) {
            for (int i = tid; i < m; i += 256) {
                double a = Wb[(int64_t)k * ld + i];
                Wb[(int64_t)k * ld + i] = Wb[(int64_t)piv * ld + i];
                Wb[(int64_t)piv * ld + i] = a;
            }
            if (tid == 0) {
                double t = cn[k]; cn[k] = cn[piv]; cn[piv] = t;
                t = cn0[k]; cn0[k] = cn0[piv]; cn0[piv] = t;
                int q = perm[k]; perm[k] = perm[piv]; perm[piv] = q;
            }
        }
        __syncthreads();
        // 2. exact norm of the pivot column below the diagonal
        double s = 0.0;
        for (int i = k + tid; i < m; i += 256) {
            double a = Wb[(int64_t)k * ld + i];
            s = fma(a, a, s);
        }
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red_v[warp] = s;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < 8; ++w) t += red_v[w];
            s_nx = sqrt(t);
        }
        __syncthreads();
        const double nx = s_nx;
        if (k == 0) R11 = nx;
        if (nx == 0.0 || nx < tol * R11) { rank = k; break; }
        // 3. reflector
        const double alpha = Wb[(int64_t)k * ld + k];
        const double beta = alpha >= 0.0 ? -nx : nx;
        const double scale = 1.0 / (alpha - beta);
        const double tk = (beta - alpha) / beta;
        for (int i = k + 1 + tid; i < m; i += 256) Wb[(int64_t)k * ld + i] *= scale;
        __syncthreads();
        if (tid == 0) {
            Wb[(int64_t)k * ld + k] = beta;
            tau[B.coff + k] = tk;
        }
        // 4. trailing update and norm downdate, one warp per column
        const double *v = Wb + (int64_t)k * ld;
        for (int c = k + 1 + warp; c < K; c += 8) {
            double *a = Wb + (int64_t)c * ld;
            double d = 0.0;
            for (int i = k + 1 + lane; i < m; i += 32) d = fma(v[i], a[i], d);
            for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            const double akc = a[k];
            d = tk * (akc + d);
            for (int i = k + 1 + lane; i < m; i += 32) a[i] = fma(-d, v[i], a[i]);
            const double rkc = akc - d;
            __syncwarp();
            if (lane == 0) a[k] = rkc;
            double cc = cn[c];
            int recompute = 0;
            if (cc != 0.0) {
                double t = fabs(rkc) / cc;
                t = (1.0 + t) * (1.0 - t);
                t = t < 0.0 ? 0.0 : t;
                double r = cc / cn0[c];
                if (t * r * r <= tol3z) recompute = 1;
                else cc = cc * sqrt(t);
            }
            if (recompute) {
                double e = 0.0;
                for (int i = k + 1 + lane; i < m; i += 32) e = fma(a[i], a[i], e);
                for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
                cc = sqrt(e);
                if (lane == 0) cn0[c] = cc;
            }
            if (lane == 0) cn[c] = cc;
        }
        __syncthreads();
    }
    if (tid == 0) {
        rank_out[blockIdx.x] = rank;
        r11_out[blockIdx.x] = R11;
    }
    for (int c = tid; c < K; c += 256) perm_out[B.coff + c] = perm[c];
}

// Kept columns of the original block, compacted: Op[:, c] = M[:, perm[c]] (FP64).
template <typename TM>
__global__ void __launch_bounds__(256) k_gather_kept(const BlkRec *__restrict__ blks, const TM *__restrict__ M,
                                                     const int32_t *__restrict__ perm, const int32_t *__restrict__ rank,
                                                     double *__restrict__ Op) {
    const BlkRec &B = blks[blockIdx.x];
    const int r = rank[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = warp; c < r; c += 8) {
        const TM *src = M + B.moff + (int64_t)perm[B.coff + c] * B.ldm;
        double *dst = Op + B.moff + (int64_t)c * B.ldm;
        for (int i = lane; i < B.m; i += 32) dst[i] = (double)src[i];
    }
}

// Q_hat = H_0 ... H_{r-1} [I_r; 0] in FP64 (Proposition 3.1), accumulated
// backwards so that H_k only touches rows >= k and columns >= k.  Optionally
// rounded to FP32 into Q32.
__global__ void __launch_bounds__(256) k_form_q(const BlkRec *__restrict__ blks, const double *__restrict__ W,
                                                const double *__restrict__ tau, const int32_t *__restrict__ rank,
                                                double *__restrict__ Q, float *__restrict__ Q32) {
    const BlkRec &B = blks[blockIdx.x];
    const int r = rank[blockIdx.x], m = B.m, ld = B.ldm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double *Qb = Q + B.moff;
    const double *Wb = W + B.moff;
    for (int c = warp; c < r; c += 8)
        for (int i = lane; i < m; i += 32) Qb[(int64_t)c * ld + i] = (i == c) ? 1.0 : 0.0;
    __syncthreads();
    for (int k = r - 1; k >= 0; --k) {
        const double tk = tau[B.coff + k];
        const double *v = Wb + (int64_t)k * ld;
        for (int c = k + warp; c < r; c += 8) {
            double *q = Qb + (int64_t)c * ld;
            double d = 0.0;
            for (int i = k + 1 + lane; i < m; i += 32) d = fma(v[i], q[i], d);
            for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            const double qk = q[k];
            d = tk * (qk + d);
            for (int i = k + 1 + lane; i < m; i += 32) q[i] = fma(-d, v[i], q[i]);
            __syncwarp();
            if (lane == 0) q[k] = qk - d;
        }
        __syncthreads();
    }
    if (Q32) {
        float *q32 = Q32 + B.moff;
        for (int c = warp; c < r; c += 8)
            for (int i = lane; i < m; i += 32) q32[(int64_t)c * ld + i] = (float)Qb[(int64_t)c * ld + i];
    }
}

rfm_status launch_filter(const HostPlan &P, void *ws, double tol, cudaStream_t st) {
    const Layout &L = P.L;
    if (L.n_blocks == 0) return RFM_OK;
    BlkRec *dB = ws_ptr<BlkRec>(ws, L.off_blk);
    const unsigned nb = (unsigned)L.n_blocks;
    const size_t sm = (size_t)L.max_K * (2 * sizeof(double) + sizeof(int));
    double *W = ws_ptr<double>(ws, L.off_W);
    double *tau = ws_ptr<double>(ws, L.off_tau);
    int32_t *perm = ws_ptr<int32_t>(ws, L.off_perm);
    int32_t *rank = ws_ptr<int32_t>(ws, L.off_rank);
    double *r11 = ws_ptr<double>(ws, L.off_r11);
    {
    ProfScope ps("k_qrcp", st);
    if (L.asm_prec == RFM_ASM_FP32) {
        RFM_CUDA_CHECK(cudaFuncSetAttribute(k_qrcp<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_qrcp<float><<<nb, 256, sm, st>>>(dB, ws_ptr<float>(ws, L.off_M), W, tau, perm, rank, r11, tol);
    } else {
        RFM_CUDA_CHECK(cudaFuncSetAttribute(k_qrcp<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_qrcp<double><<<nb, 256, sm, st>>>(dB, ws_ptr<double>(ws, L.off_M), W, tau, perm, rank, r11, tol);
    }
    }
    RFM_CUDA_CHECK(cudaGetLastError());
    double *Op = ws_ptr<double>(ws, L.off_op);
    if (L.op == RFM_OP_AR64) {
        ProfScope ps("k_gather_kept", st);
        if (L.asm_prec == RFM_ASM_FP32)
            k_gather_kept<float><<<nb, 256, 0, st>>>(dB, ws_ptr<float>(ws, L.off_M), perm, rank, Op);
        else
            k_gather_kept<double><<<nb, 256, 0, st>>>(dB, ws_ptr<double>(ws, L.off_M), perm, rank, Op);
    } else {
        ProfScope ps("k_form_q", st);
        k_form_q<<<nb, 256, 0, st>>>(dB, W, tau, rank, Op, L.op == RFM_OP_Q32 ? ws_ptr<float>(ws, L.off_q32) : nullptr);
    }
    RFM_CUDA_CHECK(cudaGetLastError());
    return RFM_OK;
}

}  // namespace rfm
