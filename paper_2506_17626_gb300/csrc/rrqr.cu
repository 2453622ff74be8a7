// rrqr.cu -- local sigma-RRQR filtering (Algorithm 1) and the operator blocks
// of the right preconditioner (Sec. 3.2, Proposition 3.1).
//
// k_qrcp: one CTA per block, FP64 Householder QR with column pivoting on a
// working copy W of M_j (column-major, leading dimension ldm).  Step k:
//   1. pivot = trailing column of largest norm (squared norms kept in shared
//      memory and compared as integers -- non-negative doubles order like
//      their bit patterns; ties to the lowest original index), swapped into
//      place;
//   2. ||W[k:m, k]|| recomputed exactly; stop when it is 0 or < tol |R_11|;
//   3. reflector beta = -sign(alpha) ||x||, v = x / (alpha - beta), v_0 = 1,
//      tau = (beta - alpha) / beta (v stored below the diagonal);
//   4. every trailing column c: W[k:m, c] -= tau v (v^T W[k:m, c]) (one warp
//      per column), applied with the unscaled x: with g = tau / (alpha - beta)
//      = -1 / beta, d = tau W[k, c] + g x^T W[k+1:m, c] and W[k+1:m, c] -=
//      (d / (alpha - beta)) x; then its squared norm is downdated,
//      ||W[k+1:m, c]||^2 = ||W[k:m, c]||^2 - W[k, c]^2, and recomputed exactly
//      when cancellation has eaten more than half the digits since the last
//      exact value (the downdated value's relative error grows like
//      eps (squared norm at last recompute / current squared norm)).
// FP64 throughput is the bound: per element of the trailing matrix one FMA
// for the dot product and one for the update.  GB300 issues an FP64 warp
// instruction at a small fraction of the FP32 rate, so the per-step scalars
// are formed once, by one warp, and comparisons avoid the FP64 pipe.
#include <cooperative_groups.h>

#include <climits>
#include <type_traits>
#include <mutex>
#include <vector>

#include "df.cuh"
#include "device.cuh"
#include "prof.cuh"

namespace rfm {

constexpr unsigned kFull = 0xffffffffu;

// Pivot order: larger squared norm first, then lower original column index.
__device__ inline long long norm_key(double c2) { return __double_as_longlong(c2); }   // c2 >= 0
__device__ inline bool key_better(long long k1, int o1, long long k2, int o2) {
    return k1 > k2 || (k1 == k2 && o1 < o2);
}

// Householder scalars of a pivot column with first entry alpha and norm
// nx > 0: beta = -sign(alpha) nx, sc = 1 / (alpha - beta) (the scaling of v),
// tau = (beta - alpha) / beta and g = tau sc = -1 / beta, from one division
// (|alpha - beta| = |alpha| + nx, so nothing cancels).
__device__ inline void house_scalars(double alpha, double nx, double *h) {
    const double beta = alpha >= 0.0 ? -nx : nx;
    const double amb = alpha - beta;
    const double inv = 1.0 / (amb * beta);
    const double g = -amb * inv;
    h[1] = beta;
    h[2] = beta * inv;   // sc
    h[3] = amb * g;      // tau
    h[4] = g;
}

// Squared-norm downdate of a trailing column after step k (rk = R(k, c)).
// Returns true when the column's norm must be recomputed exactly.
__device__ inline bool downdate(double c2, double thr, double rk, double *c2_new) {
    if (c2 == 0.0) {
        *c2_new = 0.0;
        return false;
    }
    *c2_new = fma(-rk, rk, c2);
    return !(*c2_new > thr);
}

template <typename TM, int NW>
__global__ void __launch_bounds__(NW * 32) k_qrcp(const BlkRec *__restrict__ blks, const TM *__restrict__ M,
                                              double *__restrict__ W, double *__restrict__ tau,
                                              int32_t *__restrict__ perm_out, int32_t *__restrict__ rank_out,
                                              double *__restrict__ r11_out, double tol) {
    extern __shared__ double smem[];
    const BlkRec B = blks[blockIdx.x];
    const int m = B.m, K = B.K, ld = B.ldm;
    double *cn2 = smem;            // K squared trailing norms
    double *thr = smem + K;        // K recompute thresholds: tol3z * last exact squared norm
    int *perm = (int *)(smem + 2 * K);
    constexpr int NT = NW * 32;
    __shared__ long long red_k[NW];
    __shared__ int red_o[NW], red_c[NW];
    __shared__ double s_red[NW];
    __shared__ double s_h[5];
    __shared__ int s_piv;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double *Wb = W + B.moff;
    const TM *Mb = M + B.moff;
    const double tol3z = sqrt(2.220446049250313e-16);

    // working copy in FP64
    for (int c = warp; c < K; c += NW)
        for (int i = lane; i < m; i += 32) Wb[(int64_t)c * ld + i] = (double)Mb[(int64_t)c * ld + i];
    __syncthreads();
    for (int c = warp; c < K; c += NW) {
        double s = 0.0;
        for (int i = lane; i < m; i += 32) {
            double a = Wb[(int64_t)c * ld + i];
            s = fma(a, a, s);
        }
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
        if (lane == 0) {
            cn2[c] = s;
            thr[c] = tol3z * s;
            perm[c] = c;
        }
    }
    __syncthreads();

    const int steps = m < K ? m : K;
    double R11 = 0.0;
    int rank = steps;
    for (int k = 0; k < steps; ++k) {
        // 1. pivot
        long long bk = -1;
        int bo = INT_MAX, bc = k;
        for (int c = k + tid; c < K; c += NT) {
            const long long kc = norm_key(cn2[c]);
            if (key_better(kc, perm[c], bk, bo)) { bk = kc; bo = perm[c]; bc = c; }
        }
        for (int o = 16; o; o >>= 1) {
            const long long k2 = __shfl_xor_sync(kFull, bk, o);
            const int o2 = __shfl_xor_sync(kFull, bo, o), c2 = __shfl_xor_sync(kFull, bc, o);
            if (key_better(k2, o2, bk, bo)) { bk = k2; bo = o2; bc = c2; }
        }
        if (lane == 0) { red_k[warp] = bk; red_o[warp] = bo; red_c[warp] = bc; }
        __syncthreads();
        if (tid == 0) {
            long long v = red_k[0];
            int o = red_o[0], c = red_c[0];
            for (int w = 1; w < NW; ++w)
                if (key_better(red_k[w], red_o[w], v, o)) { v = red_k[w]; o = red_o[w]; c = red_c[w]; }
            s_piv = c;
        }
        __syncthreads();
        const int piv = s_piv;
        if (piv != k) {
            for (int i = tid; i < m; i += NT) {
                double a = Wb[(int64_t)k * ld + i];
                Wb[(int64_t)k * ld + i] = Wb[(int64_t)piv * ld + i];
                Wb[(int64_t)piv * ld + i] = a;
            }
            if (tid == 0) {
                double t = cn2[k]; cn2[k] = cn2[piv]; cn2[piv] = t;
                t = thr[k]; thr[k] = thr[piv]; thr[piv] = t;
                int q = perm[k]; perm[k] = perm[piv]; perm[piv] = q;
            }
        }
        __syncthreads();
        // 2. exact norm of the pivot column below the diagonal, reflector scalars
        double s = 0.0;
        for (int i = k + tid; i < m; i += NT) {
            double a = Wb[(int64_t)k * ld + i];
            s = fma(a, a, s);
        }
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
        if (lane == 0) s_red[warp] = s;
        __syncthreads();
        if (warp == 0) {
            double t = lane < NW ? s_red[lane] : 0.0;
            for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
            if (lane == 0) {
                const double nx = sqrt(t);
                s_h[0] = nx;
                if (nx > 0.0) house_scalars(Wb[(int64_t)k * ld + k], nx, s_h);
            }
        }
        __syncthreads();
        const double nx = s_h[0];
        if (k == 0) R11 = nx;
        if (nx == 0.0 || nx < tol * R11) { rank = k; break; }
        const double sc = s_h[2], tk = s_h[3], g = s_h[4];
        // 3./4. trailing update with the unscaled pivot column, norm downdate
        const double *x = Wb + (int64_t)k * ld;
        for (int c = k + 1 + warp; c < K; c += NW) {
            double *a = Wb + (int64_t)c * ld;
            double dot = 0.0;
            for (int i = k + 1 + lane; i < m; i += 32) dot = fma(x[i], a[i], dot);
            for (int o = 16; o; o >>= 1) dot += __shfl_xor_sync(kFull, dot, o);
            const double akc = a[k];
            const double d = fma(g, dot, tk * akc);
            const double e = d * sc;
            for (int i = k + 1 + lane; i < m; i += 32) a[i] = fma(-e, x[i], a[i]);
            const double rkc = akc - d;
            __syncwarp();
            double c2;
            const bool again = downdate(cn2[c], thr[c], rkc, &c2);
            if (again) {
                double q = 0.0;
                for (int i = k + 1 + lane; i < m; i += 32) q = fma(a[i], a[i], q);
                for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(kFull, q, o);
                c2 = q;
            }
            if (lane == 0) {
                a[k] = rkc;
                cn2[c] = c2;
                if (again) thr[c] = tol3z * c2;
            }
        }
        __syncthreads();
        // v = x / (alpha - beta) below the diagonal, beta on it
        for (int i = k + 1 + tid; i < m; i += NT) Wb[(int64_t)k * ld + i] *= sc;
        if (tid == 0) {
            Wb[(int64_t)k * ld + k] = s_h[1];
            tau[B.coff + k] = tk;
        }
    }
    if (tid == 0) {
        rank_out[blockIdx.x] = rank;
        r11_out[blockIdx.x] = R11;
    }
    for (int c = tid; c < K; c += NT) perm_out[B.coff + c] = perm[c];
}

// Double-float variant of k_qrcp for FP32-assembled blocks (the global-memory
// counterpart of k_qrcp_cluster_df): the same steps in the same order, the
// working copy, norms and reflector scalars as double-floats (pairs of FP32
// numbers, 48 bits, on the FP32 pipe, `df.cuh`) held in the W arena (a
// double-float takes the 8 bytes of a double), the pivot column staged in
// shared memory.  At the end every element is converted to FP64 in place, so
// W, tau, the permutation and R leave in the layout of k_qrcp.
__device__ inline float2 dfg_in(float x) { return make_float2(x, 0.f); }
__device__ inline float2 dfg_in(double x) { return df_from_double(x); }
__device__ inline long long dfg_key(float2 c2) {   // order-preserving key of a normalised h >= 0
    unsigned lo = __float_as_uint(c2.y);
    lo = (lo & 0x80000000u) ? ~lo : (lo | 0x80000000u);
    return ((long long)__float_as_int(c2.x) << 32) | (long long)lo;
}

template <typename TM, int NW>
__global__ void __launch_bounds__(NW * 32) k_qrcp_gdf(const BlkRec *__restrict__ blks, const TM *__restrict__ M,
                                                      double *__restrict__ W, double *__restrict__ tau,
                                                      int32_t *__restrict__ perm_out, int32_t *__restrict__ rank_out,
                                                      double *__restrict__ r11_out, double tol) {
    constexpr int NT = NW * 32;
    extern __shared__ __align__(16) unsigned char gsm[];
    const BlkRec B = blks[blockIdx.x];
    const int m = B.m, K = B.K, ld = B.ldm;
    float2 *xs = reinterpret_cast<float2 *>(gsm);        // m: the pivot column of the step
    float2 *cn2 = xs + m;                                // K squared trailing norms
    float *thr = reinterpret_cast<float *>(cn2 + K);     // K recompute thresholds
    int *perm = reinterpret_cast<int *>(thr + K);        // K
    __shared__ long long red_k[NW];
    __shared__ int red_o[NW], red_c[NW];
    __shared__ float2 s_red[NW];
    __shared__ float2 s_h[4];      // beta, sc, g, tau of the step
    __shared__ double s_nx, s_tau;
    __shared__ int s_piv;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 *Wb = reinterpret_cast<float2 *>(W + B.moff);
    const TM *Mb = M + B.moff;
    const float tol3z = 1.4901161193847656e-08f;   // sqrt of the FP64 epsilon, as in the FP64 kernels

    for (int c = warp; c < K; c += NW) {
        float sh = 0.f, sl = 0.f;
        for (int i = lane; i < m; i += 32) {
            const float2 a = dfg_in(Mb[(int64_t)c * ld + i]);
            Wb[(int64_t)c * ld + i] = a;
            df_acc(a, a, sh, sl);
        }
        float2 s2 = make_float2(sh, sl);
        for (int o = 16; o; o >>= 1) s2 = df_xor_add(s2, o);
        if (lane == 0) {
            cn2[c] = s2;
            thr[c] = tol3z * s2.x;
            perm[c] = c;
        }
    }
    __syncthreads();

    const int steps = m < K ? m : K;
    double R11 = 0.0;
    int rank = steps;
    for (int k = 0; k < steps; ++k) {
        // 1. pivot: the trailing column of largest squared norm, ties to the lowest original index
        long long bk = -1;
        int bo = INT_MAX, bc = k;
        for (int c = k + tid; c < K; c += NT) {
            const long long kc = dfg_key(cn2[c]);
            if (key_better(kc, perm[c], bk, bo)) { bk = kc; bo = perm[c]; bc = c; }
        }
        for (int o = 16; o; o >>= 1) {
            const long long k2 = __shfl_xor_sync(kFull, bk, o);
            const int o2 = __shfl_xor_sync(kFull, bo, o), c2 = __shfl_xor_sync(kFull, bc, o);
            if (key_better(k2, o2, bk, bo)) { bk = k2; bo = o2; bc = c2; }
        }
        if (lane == 0) { red_k[warp] = bk; red_o[warp] = bo; red_c[warp] = bc; }
        __syncthreads();
        if (tid == 0) {
            long long v = red_k[0];
            int o = red_o[0], c = red_c[0];
            for (int w = 1; w < NW; ++w)
                if (key_better(red_k[w], red_o[w], v, o)) { v = red_k[w]; o = red_o[w]; c = red_c[w]; }
            s_piv = c;
        }
        __syncthreads();
        const int piv = s_piv;
        if (piv != k) {
            for (int i = tid; i < m; i += NT) {
                const float2 a = Wb[(int64_t)k * ld + i];
                Wb[(int64_t)k * ld + i] = Wb[(int64_t)piv * ld + i];
                Wb[(int64_t)piv * ld + i] = a;
            }
            if (tid == 0) {
                const float2 t = cn2[k]; cn2[k] = cn2[piv]; cn2[piv] = t;
                const float u = thr[k]; thr[k] = thr[piv]; thr[piv] = u;
                const int q = perm[k]; perm[k] = perm[piv]; perm[piv] = q;
            }
        }
        __syncthreads();
        // 2. the pivot column (rows k..m) to shared memory, its exact norm, reflector scalars
        {
            float sh = 0.f, sl = 0.f;
            for (int i = k + tid; i < m; i += NT) {
                const float2 x = Wb[(int64_t)k * ld + i];
                xs[i] = x;
                df_acc(x, x, sh, sl);
            }
            float2 s2 = make_float2(sh, sl);
            for (int o = 16; o; o >>= 1) s2 = df_xor_add(s2, o);
            if (lane == 0) s_red[warp] = s2;
        }
        __syncthreads();
        if (warp == 0) {
            float2 t = lane < NW ? s_red[lane] : make_float2(0.f, 0.f);
            for (int o = 16; o; o >>= 1) t = df_xor_add(t, o);
            if (lane == 0) {
                const float2 nxd = t.x > 0.f ? df_sqrt(t) : make_float2(0.f, 0.f);
                s_nx = df_to_double(nxd);
                if (nxd.x > 0.f) {
                    const float2 alpha = xs[k];
                    const float2 beta = alpha.x >= 0.f ? df_neg(nxd) : nxd;
                    const float2 amb = df_sub(alpha, beta);
                    const float2 inv = df_rcp(df_mul(amb, beta));
                    const float2 g = df_neg(df_mul(amb, inv));
                    const float2 tk = df_mul(amb, g);
                    s_h[0] = beta;
                    s_h[1] = df_mul(beta, inv);
                    s_h[2] = g;
                    s_h[3] = tk;
                    s_tau = df_to_double(tk);
                }
            }
        }
        __syncthreads();
        const double nx = s_nx;
        if (k == 0) R11 = nx;
        if (nx == 0.0 || nx < tol * R11) { rank = k; break; }
        const float2 sc = s_h[1], g = s_h[2], tk = s_h[3];
        // 3. trailing update with the unscaled pivot column, norm downdate
        for (int c = k + 1 + warp; c < K; c += NW) {
            float2 *a = Wb + (int64_t)c * ld;
            float ph = 0.f, pl = 0.f;
            for (int i = k + 1 + lane; i < m; i += 32) df_acc(xs[i], a[i], ph, pl);
            float2 dot = make_float2(ph, pl);
            for (int o = 16; o; o >>= 1) dot = df_xor_add(dot, o);
            const float2 akc = a[k];
            const float2 d = df_add(df_mul(g, dot), df_mul(tk, akc));
            const float2 e = df_mul(d, sc);
            for (int i = k + 1 + lane; i < m; i += 32) a[i] = df_axmy(a[i], e, xs[i]);
            const float2 rkc = df_sub(akc, d);
            __syncwarp();
            const float2 c2o = cn2[c];
            float2 c2 = make_float2(0.f, 0.f);
            bool again = false;
            if (c2o.x != 0.f) {
                c2 = df_sub(c2o, df_mul(rkc, rkc));
                again = !(c2.x > thr[c]);
            }
            if (again) {
                float qh = 0.f, ql = 0.f;
                for (int i = k + 1 + lane; i < m; i += 32) df_acc(a[i], a[i], qh, ql);
                float2 q = make_float2(qh, ql);
                for (int o = 16; o; o >>= 1) q = df_xor_add(q, o);
                c2 = q;
            }
            if (lane == 0) {
                a[k] = rkc;
                cn2[c] = c2;
                if (again) thr[c] = tol3z * c2.x;
            }
        }
        __syncthreads();
        // v = x sc below the diagonal, beta on it
        for (int i = k + 1 + tid; i < m; i += NT) Wb[(int64_t)k * ld + i] = df_mul(xs[i], sc);
        if (tid == 0) {
            Wb[(int64_t)k * ld + k] = s_h[0];
            tau[B.coff + k] = s_tau;
        }
        __syncthreads();
    }
    __syncthreads();
    // the layout of k_qrcp: every element to FP64 in place (same 8 bytes, same thread)
    for (int c = warp; c < K; c += NW)
        for (int i = lane; i < m; i += 32) {
            const float2 v = Wb[(int64_t)c * ld + i];
            W[B.moff + (int64_t)c * ld + i] = df_to_double(v);
        }
    if (tid == 0) {
        rank_out[blockIdx.x] = rank;
        r11_out[blockIdx.x] = R11;
    }
    for (int c = tid; c < K; c += NT) perm_out[B.coff + c] = perm[c];
}

// k_qrcp_gdf with the trailing update deferred over panels of NB steps (the
// BLAS-3 QR with column pivoting of Quintana-Orti, Sun and Bischof 1998):
// within a panel the trailing columns keep their values from the panel's
// start, A0, and the updated matrix is A0 - V F^T, with V the panel's
// reflectors (v_j: 1 at its step's row, v below) and F[c][j] = tau_j
// (A_j^T v_j)[c], A_j the matrix after the panel's first j steps.  Step k =
// k0 + j:
//   pivot from the downdated squared norms (as k_qrcp_gdf); the pivot column
//     updated, x = A0[k:, k] - V[k:, 0:j] F[k, 0:j]^T, and its reflector;
//   y = V[k:, 0:j]^T v_j, then per trailing column c: one read pass for
//     A0[k:, c]^T v_j, F[c][j] = tau_j (that - F[c, 0:j] y), the row-k entry
//     r_kc = A0[k][c] - V[k, 0:j] F[c, 0:j]^T - F[c][j] (an entry of R, stored
//     in place), and the norm downdate ||a_c||^2 -= r_kc^2 with the same
//     recompute rule (the recomputed norm from the updated column);
// after the panel, one pass A0[k0+nb:, c] -= V[k0+nb:, :] F[c, :]^T per
// trailing column.  Per panel of nb steps each trailing column is read nb
// times and read and written once, against nb times each in k_qrcp_gdf.
// Shared memory: V (NB x ld double-floats), F (K x NB), the norms, the
// recompute thresholds and the permutation.
template <typename TM, int NW, int NB>
__global__ void __launch_bounds__(NW * 32) k_qrcp_gdf_blk(const BlkRec *__restrict__ blks, const TM *__restrict__ M,
                                                          double *__restrict__ W, double *__restrict__ tau,
                                                          int32_t *__restrict__ perm_out, int32_t *__restrict__ rank_out,
                                                          double *__restrict__ r11_out, double tol) {
    constexpr int NT = NW * 32;
    extern __shared__ __align__(16) unsigned char gsm[];
    const BlkRec B = blks[blockIdx.x];
    const int m = B.m, K = B.K, ld = B.ldm;
    float2 *Vs = reinterpret_cast<float2 *>(gsm);        // NB x ld: v_j at Vs[j * ld + i], rows >= its step
    float2 *Fs = Vs + (size_t)NB * ld;                   // K x NB: F[c][j] at Fs[c * NB + j]
    float2 *cn2 = Fs + (size_t)K * NB;                   // K squared trailing norms
    float *thr = reinterpret_cast<float *>(cn2 + K);     // K recompute thresholds
    int *perm = reinterpret_cast<int *>(thr + K);        // K
    __shared__ long long red_k[NW];
    __shared__ int red_o[NW], red_c[NW];
    __shared__ float2 s_red[NW];
    __shared__ float2 s_h[4];      // beta, sc, g, tau of the step
    __shared__ float2 s_y[NB];     // V[k:, 0:j]^T v_j
    __shared__ double s_nx, s_tau;
    __shared__ int s_piv;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 *Wb = reinterpret_cast<float2 *>(W + B.moff);
    const TM *Mb = M + B.moff;
    const float tol3z = 1.4901161193847656e-08f;   // sqrt of the FP64 epsilon, as in the FP64 kernels

    for (int c = warp; c < K; c += NW) {
        float sh = 0.f, sl = 0.f;
        for (int i = lane; i < m; i += 32) {
            const float2 a = dfg_in(Mb[(int64_t)c * ld + i]);
            Wb[(int64_t)c * ld + i] = a;
            df_acc(a, a, sh, sl);
        }
        float2 s2 = make_float2(sh, sl);
        for (int o = 16; o; o >>= 1) s2 = df_xor_add(s2, o);
        if (lane == 0) {
            cn2[c] = s2;
            thr[c] = tol3z * s2.x;
            perm[c] = c;
        }
    }
    for (int e = tid; e < K * NB; e += NT) Fs[e] = make_float2(0.f, 0.f);
    __syncthreads();

    const int steps = m < K ? m : K;
    double R11 = 0.0;
    int rank = steps;
    bool stop = false;
    for (int k0 = 0; k0 < steps && !stop; k0 += NB) {
        const int nbp = min(NB, steps - k0);
        int j = 0;
        for (; j < nbp; ++j) {
            const int k = k0 + j;
            // 1. pivot: the trailing column of largest squared norm, ties to the lowest original index
            long long bk = -1;
            int bo = INT_MAX, bc = k;
            for (int c = k + tid; c < K; c += NT) {
                const long long kc = dfg_key(cn2[c]);
                if (key_better(kc, perm[c], bk, bo)) { bk = kc; bo = perm[c]; bc = c; }
            }
            for (int o = 16; o; o >>= 1) {
                const long long k2 = __shfl_xor_sync(kFull, bk, o);
                const int o2 = __shfl_xor_sync(kFull, bo, o), c2 = __shfl_xor_sync(kFull, bc, o);
                if (key_better(k2, o2, bk, bo)) { bk = k2; bo = o2; bc = c2; }
            }
            if (lane == 0) { red_k[warp] = bk; red_o[warp] = bo; red_c[warp] = bc; }
            __syncthreads();
            if (tid == 0) {
                long long v = red_k[0];
                int o = red_o[0], c = red_c[0];
                for (int w = 1; w < NW; ++w)
                    if (key_better(red_k[w], red_o[w], v, o)) { v = red_k[w]; o = red_o[w]; c = red_c[w]; }
                s_piv = c;
            }
            __syncthreads();
            const int piv = s_piv;
            if (piv != k) {   // whole columns (R entries above, panel-start values below) with their F rows
                for (int i = tid; i < m; i += NT) {
                    const float2 a = Wb[(int64_t)k * ld + i];
                    Wb[(int64_t)k * ld + i] = Wb[(int64_t)piv * ld + i];
                    Wb[(int64_t)piv * ld + i] = a;
                }
                if (tid < NB) {
                    const float2 f = Fs[k * NB + tid];
                    Fs[k * NB + tid] = Fs[piv * NB + tid];
                    Fs[piv * NB + tid] = f;
                }
                if (tid == 0) {
                    const float2 t = cn2[k]; cn2[k] = cn2[piv]; cn2[piv] = t;
                    const float u = thr[k]; thr[k] = thr[piv]; thr[piv] = u;
                    const int q = perm[k]; perm[k] = perm[piv]; perm[piv] = q;
                }
            }
            __syncthreads();
            // 2. the updated pivot column (rows k..m) into V's slot j, its exact norm, reflector scalars
            {
                float2 fk[NB];
#pragma unroll
                for (int jj = 0; jj < NB; ++jj) fk[jj] = Fs[k * NB + jj];
                float sh = 0.f, sl = 0.f;
                for (int i = k + tid; i < m; i += NT) {
                    float2 x = Wb[(int64_t)k * ld + i];
                    if (j > 0) {
                        float h = 0.f, l = 0.f;
#pragma unroll
                        for (int jj = 0; jj < NB; ++jj)
                            if (jj < j) df_acc(Vs[jj * ld + i], fk[jj], h, l);
                        x = df_sub(x, df_add(make_float2(h, 0.f), make_float2(l, 0.f)));
                    }
                    Vs[j * ld + i] = x;
                    df_acc(x, x, sh, sl);
                }
                float2 s2 = make_float2(sh, sl);
                for (int o = 16; o; o >>= 1) s2 = df_xor_add(s2, o);
                if (lane == 0) s_red[warp] = s2;
            }
            __syncthreads();
            if (warp == 0) {
                float2 t = lane < NW ? s_red[lane] : make_float2(0.f, 0.f);
                for (int o = 16; o; o >>= 1) t = df_xor_add(t, o);
                if (lane == 0) {
                    const float2 nxd = t.x > 0.f ? df_sqrt(t) : make_float2(0.f, 0.f);
                    s_nx = df_to_double(nxd);
                    if (nxd.x > 0.f) {
                        const float2 alpha = Vs[j * ld + k];
                        const float2 beta = alpha.x >= 0.f ? df_neg(nxd) : nxd;
                        const float2 amb = df_sub(alpha, beta);
                        const float2 inv = df_rcp(df_mul(amb, beta));
                        const float2 g = df_neg(df_mul(amb, inv));
                        const float2 tk = df_mul(amb, g);
                        s_h[0] = beta;
                        s_h[1] = df_mul(beta, inv);
                        s_h[2] = g;
                        s_h[3] = tk;
                        s_tau = df_to_double(tk);
                    }
                }
            }
            __syncthreads();
            const double nx = s_nx;
            if (k == 0) R11 = nx;
            if (nx == 0.0 || nx < tol * R11) { rank = k; stop = true; break; }
            const float2 sc = s_h[1], tk = s_h[3];
            // 3. v_j = x sc below the diagonal (1 on it) in V and in the block, beta on the diagonal
            for (int i = k + 1 + tid; i < m; i += NT) {
                const float2 v = df_mul(Vs[j * ld + i], sc);
                Vs[j * ld + i] = v;
                Wb[(int64_t)k * ld + i] = v;
            }
            if (tid == 0) {
                Vs[j * ld + k] = make_float2(1.f, 0.f);
                Wb[(int64_t)k * ld + k] = s_h[0];
                tau[B.coff + k] = s_tau;
            }
            __syncthreads();
            // 4. y = V[k:, 0:j]^T v_j
            for (int jj = warp; jj < j; jj += NW) {
                float h = 0.f, l = 0.f;
                for (int i = k + lane; i < m; i += 32) df_acc(Vs[jj * ld + i], Vs[j * ld + i], h, l);
                float2 d = make_float2(h, l);
                for (int o = 16; o; o >>= 1) d = df_xor_add(d, o);
                if (lane == 0) s_y[jj] = d;
            }
            __syncthreads();
            // 5. trailing columns: F[c][j], the row-k entry (of R), the norm downdate
            float2 yv[NB], vk[NB];
#pragma unroll
            for (int jj = 0; jj < NB; ++jj) {
                yv[jj] = jj < j ? s_y[jj] : make_float2(0.f, 0.f);
                vk[jj] = jj < j ? Vs[jj * ld + k] : make_float2(0.f, 0.f);
            }
            for (int c = k + 1 + warp; c < K; c += NW) {
                float2 *a = Wb + (int64_t)c * ld;
                float ph = 0.f, pl = 0.f;
                for (int i = k + lane; i < m; i += 32) df_acc(Vs[j * ld + i], a[i], ph, pl);
                float2 dot = make_float2(ph, pl);
                for (int o = 16; o; o >>= 1) dot = df_xor_add(dot, o);
                float2 fr[NB];
#pragma unroll
                for (int jj = 0; jj < NB; ++jj) fr[jj] = Fs[c * NB + jj];
                float h = 0.f, l = 0.f;
#pragma unroll
                for (int jj = 0; jj < NB; ++jj)
                    if (jj < j) df_acc(fr[jj], yv[jj], h, l);
                const float2 fcj = df_mul(tk, df_sub(dot, df_add(make_float2(h, 0.f), make_float2(l, 0.f))));
                h = 0.f;
                l = 0.f;
#pragma unroll
                for (int jj = 0; jj < NB; ++jj)
                    if (jj < j) df_acc(vk[jj], fr[jj], h, l);
                const float2 akc = a[k];
                const float2 rkc = df_sub(df_sub(akc, df_add(make_float2(h, 0.f), make_float2(l, 0.f))), fcj);
                __syncwarp();
                const float2 c2o = cn2[c];
                float2 c2 = make_float2(0.f, 0.f);
                bool again = false;
                if (c2o.x != 0.f) {
                    c2 = df_sub(c2o, df_mul(rkc, rkc));
                    again = !(c2.x > thr[c]);
                }
                if (again) {   // the updated column below row k, formed on the fly
                    float qh = 0.f, ql = 0.f;
                    for (int i = k + 1 + lane; i < m; i += 32) {
                        float uh = 0.f, ul = 0.f;
#pragma unroll
                        for (int jj = 0; jj < NB; ++jj)
                            if (jj < j) df_acc(Vs[jj * ld + i], fr[jj], uh, ul);
                        df_acc(Vs[j * ld + i], fcj, uh, ul);
                        const float2 u = df_sub(a[i], df_add(make_float2(uh, 0.f), make_float2(ul, 0.f)));
                        df_acc(u, u, qh, ql);
                    }
                    float2 q = make_float2(qh, ql);
                    for (int o = 16; o; o >>= 1) q = df_xor_add(q, o);
                    c2 = q;
                }
                if (lane == 0) {
                    Fs[c * NB + j] = fcj;
                    a[k] = rkc;
                    cn2[c] = c2;
                    if (again) thr[c] = tol3z * c2.x;
                }
            }
            __syncthreads();
        }
        if (stop) break;
        // 6. the panel's update of the trailing columns below its rows, A0 -= V F^T
        const int kend = k0 + nbp;
        for (int c = kend + warp; c < K; c += NW) {
            float2 *a = Wb + (int64_t)c * ld;
            float2 fr[NB];
#pragma unroll
            for (int jj = 0; jj < NB; ++jj) fr[jj] = Fs[c * NB + jj];
            for (int i = kend + lane; i < m; i += 32) {
                float h = 0.f, l = 0.f;
#pragma unroll
                for (int jj = 0; jj < NB; ++jj)
                    if (jj < nbp) df_acc(Vs[jj * ld + i], fr[jj], h, l);
                a[i] = df_sub(a[i], df_add(make_float2(h, 0.f), make_float2(l, 0.f)));
            }
        }
        __syncthreads();
        for (int e = tid; e < (K - kend) * NB; e += NT) Fs[(size_t)kend * NB + e] = make_float2(0.f, 0.f);
        __syncthreads();
    }
    __syncthreads();
    // the layout of k_qrcp: every element to FP64 in place (same 8 bytes, same thread)
    for (int c = warp; c < K; c += NW)
        for (int i = lane; i < m; i += 32) {
            const float2 v = Wb[(int64_t)c * ld + i];
            W[B.moff + (int64_t)c * ld + i] = df_to_double(v);
        }
    if (tid == 0) {
        rank_out[blockIdx.x] = rank;
        r11_out[blockIdx.x] = R11;
    }
    for (int c = tid; c < K; c += NT) perm_out[B.coff + c] = perm[c];
}

// Q_hat = H_0 ... H_{r-1} [I_r; 0] of k_form_q in double-float arithmetic,
// for the FP32 operator (rounded to FP32 at the end): the working columns as
// double-floats in the FP64 operator arena (which the FP32 operator leaves
// free), the reflector of the step staged in shared memory.
template <int NW>
__global__ void __launch_bounds__(NW * 32) k_form_q_gdf(const BlkRec *__restrict__ blks, const double *__restrict__ W,
                                                        const double *__restrict__ tau, const int32_t *__restrict__ rank,
                                                        double *__restrict__ Q, float *__restrict__ Q32) {
    constexpr int NT = NW * 32;
    extern __shared__ __align__(16) float2 vs[];   // m: the reflector of the step
    const BlkRec &B = blks[blockIdx.x];
    const int r = rank[blockIdx.x], m = B.m, ld = B.ldm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 *Qb = reinterpret_cast<float2 *>(Q + B.moff);
    const double *Wb = W + B.moff;
    for (int c = warp; c < r; c += NW)
        for (int i = lane; i < ld; i += 32) Qb[(int64_t)c * ld + i] = make_float2((i == c && i < m) ? 1.f : 0.f, 0.f);
    __syncthreads();
    for (int k = r - 1; k >= 0; --k) {
        const float2 tk = df_from_double(tau[B.coff + k]);
        for (int i = k + 1 + tid; i < m; i += NT) vs[i] = df_from_double(Wb[(int64_t)k * ld + i]);
        __syncthreads();
        for (int c = k + warp; c < r; c += NW) {
            float2 *q = Qb + (int64_t)c * ld;
            float ph = 0.f, pl = 0.f;
            for (int i = k + 1 + lane; i < m; i += 32) df_acc(vs[i], q[i], ph, pl);
            float2 dot = make_float2(ph, pl);
            for (int o = 16; o; o >>= 1) dot = df_xor_add(dot, o);
            const float2 qk = q[k];
            const float2 d = df_mul(tk, df_add(qk, dot));
            for (int i = k + 1 + lane; i < m; i += 32) q[i] = df_axmy(q[i], d, vs[i]);
            __syncwarp();
            if (lane == 0) q[k] = df_sub(qk, d);
        }
        __syncthreads();
    }
    float *q32 = Q32 + B.moff;
    for (int c = warp; c < r; c += NW)
        for (int i = lane; i < ld; i += 32)
            q32[(int64_t)c * ld + i] = i < m ? df_to_float(Qb[(int64_t)c * ld + i]) : 0.f;
}

// The same Q_hat with NB reflectors per pass over each column (compact WY
// form, Schreiber and Van Loan 1989): H_k0 ... H_k0+nb-1 = I - V T V^T with
// V the panel's reflectors (unit at row k0 + t, zeros above) and T upper
// triangular, T[t][t] = tau_t, T[0:t, t] = -tau_t T[0:t, 0:t] (V[:, 0:t]^T
// v_t).  Going backwards over the panels, every column c >= k0 takes
// w = V^T q, z = T w, q -= V z: one read and one read-write of the column per
// panel instead of per reflector, the same arithmetic per element.  All in
// double-float; the panel (nb x (m - k0)) lives in shared memory.
template <int NW, int NB>
__global__ void __launch_bounds__(NW * 32) k_form_q_gdf_blk(const BlkRec *__restrict__ blks, const double *__restrict__ W,
                                                            const double *__restrict__ tau, const int32_t *__restrict__ rank,
                                                            double *__restrict__ Q, float *__restrict__ Q32) {
    constexpr int NT = NW * 32;
    extern __shared__ __align__(16) float2 vs[];   // NB x ld: v_t at vs[t * ld + i]
    __shared__ float2 Gs[NB][NB], Ts[NB][NB];
    const BlkRec &B = blks[blockIdx.x];
    const int r = rank[blockIdx.x], m = B.m, ld = B.ldm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 *Qb = reinterpret_cast<float2 *>(Q + B.moff);
    const double *Wb = W + B.moff;
    for (int c = warp; c < r; c += NW)
        for (int i = lane; i < ld; i += 32) Qb[(int64_t)c * ld + i] = make_float2((i == c && i < m) ? 1.f : 0.f, 0.f);
    for (int p = (r + NB - 1) / NB - 1; p >= 0; --p) {
        const int k0 = p * NB, nb = min(NB, r - k0), mr = m - k0;
        __syncthreads();   // the previous panel's columns and shared arrays are done with
        for (int e = tid; e < nb * mr; e += NT) {
            const int t = e / mr, i = k0 + e % mr;
            vs[t * ld + i] = i < k0 + t ? make_float2(0.f, 0.f)
                                        : (i == k0 + t ? make_float2(1.f, 0.f) : df_from_double(Wb[(int64_t)(k0 + t) * ld + i]));
        }
        __syncthreads();
        // G[s][t] = v_s . v_t for s < t (v_t is zero above row k0 + t), one warp per pair
        for (int pr = warp; pr < nb * nb; pr += NW) {
            const int s2 = pr / nb, t = pr % nb;
            if (s2 >= t) continue;
            float h = 0.f, l = 0.f;
            for (int i = k0 + t + lane; i < m; i += 32) df_acc(vs[s2 * ld + i], vs[t * ld + i], h, l);
            float2 d = make_float2(h, l);
            for (int o = 16; o; o >>= 1) d = df_xor_add(d, o);
            if (lane == 0) Gs[s2][t] = d;
        }
        __syncthreads();
        if (tid == 0) {
            for (int t = 0; t < nb; ++t) {
                const float2 tt = df_from_double(tau[B.coff + k0 + t]);
                for (int s2 = 0; s2 < t; ++s2) {
                    float h = 0.f, l = 0.f;
                    for (int u = s2; u < t; ++u) df_acc(Ts[s2][u], Gs[u][t], h, l);
                    Ts[s2][t] = df_neg(df_mul(tt, df_add(make_float2(h, 0.f), make_float2(l, 0.f))));
                }
                Ts[t][t] = tt;
            }
        }
        __syncthreads();
        for (int c = k0 + warp; c < r; c += NW) {
            float2 *q = Qb + (int64_t)c * ld;
            float wh[NB], wl[NB];
#pragma unroll
            for (int t = 0; t < NB; ++t) wh[t] = wl[t] = 0.f;
            for (int i = k0 + lane; i < m; i += 32) {
                const float2 qi = q[i];
#pragma unroll
                for (int t = 0; t < NB; ++t)
                    if (t < nb) df_acc(vs[t * ld + i], qi, wh[t], wl[t]);
            }
            float2 z[NB];
#pragma unroll
            for (int t = 0; t < NB; ++t) {
                float2 w = make_float2(wh[t], wl[t]);
                for (int o = 16; o; o >>= 1) w = df_xor_add(w, o);
                z[t] = w;   // w_t, every lane
            }
            // z = T w in place (upper triangular: z_s uses w_t for t >= s)
#pragma unroll
            for (int s2 = 0; s2 < NB; ++s2) {
                if (s2 >= nb) break;
                float h = 0.f, l = 0.f;
#pragma unroll
                for (int t = 0; t < NB; ++t)
                    if (t >= s2 && t < nb) df_acc(Ts[s2][t], z[t], h, l);
                z[s2] = df_add(make_float2(h, 0.f), make_float2(l, 0.f));
            }
            for (int i = k0 + lane; i < m; i += 32) {
                float h = 0.f, l = 0.f;
#pragma unroll
                for (int t = 0; t < NB; ++t)
                    if (t < nb) df_acc(vs[t * ld + i], z[t], h, l);
                q[i] = df_sub(q[i], df_add(make_float2(h, 0.f), make_float2(l, 0.f)));
            }
        }
    }
    __syncthreads();
    float *q32 = Q32 + B.moff;
    for (int c = warp; c < r; c += NW)
        for (int i = lane; i < ld; i += 32)
            q32[(int64_t)c * ld + i] = i < m ? df_to_float(Qb[(int64_t)c * ld + i]) : 0.f;
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
        for (int i = lane; i < B.ldm; i += 32) dst[i] = i < B.m ? (double)src[i] : 0.0;
    }
}

// Q_hat = H_0 ... H_{r-1} [I_r; 0] in FP64 (Proposition 3.1), accumulated
// backwards so that H_k only touches rows >= k and columns >= k.  Optionally
// rounded to FP32 into Q32.
template <int NW>
__global__ void __launch_bounds__(NW * 32) k_form_q(const BlkRec *__restrict__ blks, const double *__restrict__ W,
                                                const double *__restrict__ tau, const int32_t *__restrict__ rank,
                                                double *__restrict__ Q, float *__restrict__ Q32) {
    const BlkRec &B = blks[blockIdx.x];
    const int r = rank[blockIdx.x], m = B.m, ld = B.ldm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double *Qb = Q + B.moff;
    const double *Wb = W + B.moff;
    for (int c = warp; c < r; c += NW)
        for (int i = lane; i < ld; i += 32) Qb[(int64_t)c * ld + i] = (i == c && i < m) ? 1.0 : 0.0;
    __syncthreads();
    for (int k = r - 1; k >= 0; --k) {
        const double tk = tau[B.coff + k];
        const double *v = Wb + (int64_t)k * ld;
        for (int c = k + warp; c < r; c += NW) {
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
        for (int c = warp; c < r; c += NW)
            for (int i = lane; i < ld; i += 32) q32[(int64_t)c * ld + i] = i < m ? (float)Qb[(int64_t)c * ld + i] : 0.f;
    }
}

}  // namespace rfm

namespace rfm {
// ---------------------------------------------------------------------------
// Cluster variant: the block lives in the shared memory of a cluster of C
// CTAs (thread-block cluster, distributed shared memory), distributed by
// columns: original column c belongs to CTA c mod C, slot c / C, and never
// moves.  Pivoting retires the chosen column in place and records its
// position.  One cluster barrier and two CTA barriers per step:
//   - every warp, right after updating its trailing columns, pushes its best
//     one (squared norm as an integer key, original index) into a slot of
//     every CTA of the cluster (double-buffered by step parity);
//   - after the cluster barrier every warp reduces the C x 8 candidates in
//     its own shared memory and takes the same winner;
//   - every CTA copies the winner's column (rows k..m) through DSMEM and sums
//     its squares; one warp forms the reflector scalars (same data, same
//     order in every CTA: bit-identical), and every warp updates its own
//     trailing columns, two at a time (the two dot products reduce-scattered
//     in one shuffle tree), with the unscaled pivot column, downdating each
//     column's squared norm on the spot;
//   - the owner writes beta and the scaled v into the retired column after
//     the next cluster barrier, when no CTA can still be reading it.
// The arithmetic is that of k_qrcp step for step, so both kernels return the
// same factors.  No global memory traffic inside the factorisation.  Q_hat
// (when wanted) is then accumulated backwards in the same shared memory,
// each CTA on its own columns, prefetching the next reflector from global
// memory.
// ---------------------------------------------------------------------------
namespace cg = cooperative_groups;

struct __align__(16) Cand {
    long long key, orig;
};

constexpr int kQT = 256;          // threads of a cluster-QR CTA (measured: 512 was slower on the 2D workload)
constexpr int kQW = kQT / 32;

template <typename TM, int C>
__global__ void __launch_bounds__(kQT) k_qrcp_cluster(const BlkRec *__restrict__ blks,
                                                      const int32_t *__restrict__ order, const TM *__restrict__ M,
                                                      double *__restrict__ W, double *__restrict__ tau,
                                                      int32_t *__restrict__ perm_out, int32_t *__restrict__ rank_out,
                                                      double *__restrict__ r11_out, double tol, int nloc_max,
                                                      int ld_loc, double *__restrict__ Qout, float *__restrict__ Q32) {
    cg::cluster_group cl = cg::this_cluster();
    const int cr = (int)cl.block_rank();
    const int b = order ? order[blockIdx.x / C] : (int)(blockIdx.x / C);
    const BlkRec B = blks[b];
    const int m = B.m, K = B.K, ld = B.ldm;
    extern __shared__ __align__(16) double sm[];
    double *A = sm;                                  // nloc_max x ld_loc
    double *vbuf = A + (size_t)nloc_max * ld_loc;     // ld_loc: pivot column of even steps (later: Q prefetch)
    double *vbuf2 = vbuf + ld_loc;                   // ld_loc: pivot column of odd steps
    double *cn2 = vbuf2 + ld_loc;                    // nloc_max: squared trailing norms
    double *thr = cn2 + nloc_max;                    // nloc_max: tol3z * last exact squared norm
    int *pos = (int *)(thr + nloc_max);              // nloc_max: position of the column, -1 while trailing
    int *lives = pos + nloc_max;                     // nloc_max: slots of the trailing columns (any order)
    int *where = lives + nloc_max;                   // nloc_max: index of a slot in lives
    __shared__ Cand cands[2][C * kQW];
    __shared__ double s_red[kQW];
    __shared__ double s_h[5];    // nx, beta, sc, tau, g of the step
    __shared__ int s_ndrop;
    __shared__ int s_nlive;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nloc = (K - cr + C - 1) / C;   // columns owned by this CTA
    double *Wb = W + B.moff;
    const double tol3z = sqrt(2.220446049250313e-16);

    // lanes 0..C-1 store the warp's candidate into the same slot of every CTA
    auto push = [&](int par, long long key, int orig) {
        if (lane < C) {
            Cand *dst = cl.map_shared_rank(&cands[par][cr * kQW + warp], lane);
            *reinterpret_cast<longlong2 *>(dst) = make_longlong2(key, (long long)orig);
        }
    };
    cl.sync();   // every CTA of the cluster runs before any DSMEM access

    long long bk = -1;
    int bo = INT_MAX;
    for (int l = warp; l < nloc; l += kQW) {
        const int c = cr + C * l;
        const TM *src = M + B.moff + (int64_t)c * ld;
        double s = 0.0;
        for (int i = lane; i < m; i += 32) {
            double a = (double)src[i];
            A[(size_t)l * ld_loc + i] = a;
            s = fma(a, a, s);
        }
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
        if (lane == 0) {
            cn2[l] = s;
            thr[l] = tol3z * s;
            pos[l] = -1;
            lives[l] = l;
            where[l] = l;
        }
        if (key_better(norm_key(s), c, bk, bo)) { bk = norm_key(s); bo = c; }
    }
    if (tid == 0) s_nlive = nloc;
    push(0, bk, bo);
    const int steps = m < K ? m : K;
    double R11 = 0.0;
    int rank = steps;
    int pend_slot = -1, pend_k = 0;   // owner's deferred write of the last reflector
    double pend_beta = 0.0, pend_sc = 0.0;
    for (int k = 0; k < steps; ++k) {
        const int par = k & 1;
        double *vb = par ? vbuf2 : vbuf;
        cl.sync();
        // 1. winner over the cluster, in every warp
        {
            bk = -1;
            bo = INT_MAX;
            for (int t = lane; t < C * kQW; t += 32) {
                const longlong2 cd = *reinterpret_cast<const longlong2 *>(&cands[par][t]);
                if (key_better(cd.x, (int)cd.y, bk, bo)) { bk = cd.x; bo = (int)cd.y; }
            }
            for (int o = 16; o; o >>= 1) {
                const long long k2 = __shfl_xor_sync(kFull, bk, o);
                const int o2 = __shfl_xor_sync(kFull, bo, o);
                if (key_better(k2, o2, bk, bo)) { bk = k2; bo = o2; }
            }
        }
        const int own = bo % C, wsl = bo / C;   // owner CTA and its slot
        // 2. deferred write of the previous reflector into its retired column
        if (pend_slot >= 0) {
            const double *vp = par ? vbuf : vbuf2;
            double *x = A + (size_t)pend_slot * ld_loc;
            for (int i = pend_k + 1 + tid; i < m; i += kQT) x[i] = vp[i] * pend_sc;
            if (tid == 0) x[pend_k] = pend_beta;
            pend_slot = -1;
        }
        if (cr == own && tid == 0) {
            pos[wsl] = k;
            // retire the pivot slot from the trailing list (swap with the last)
            const int at = where[wsl], last = lives[s_nlive - 1];
            lives[at] = last;
            where[last] = at;
            s_nlive -= 1;
        }
        // 3. copy the pivot column (rows k..m) from its owner, sum of squares
        {
            const double *rx = cl.map_shared_rank(A, own) + (size_t)wsl * ld_loc;
            double s = 0.0;
            for (int i = k + tid; i < m; i += kQT) {
                const double x = rx[i];
                vb[i] = x;
                s = fma(x, x, s);
            }
            for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
            if (lane == 0) s_red[warp] = s;
        }
        __syncthreads();
        // 4. exact norm and reflector scalars (one warp)
        if (warp == 0) {
            double t = lane < kQW ? s_red[lane] : 0.0;
            for (int o = kQW / 2; o; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
            if (lane == 0) {
                const double nx = sqrt(t);
                s_h[0] = nx;
                if (nx > 0.0) house_scalars(vb[k], nx, s_h);
            }
        }
        __syncthreads();
        const double nx = s_h[0];
        if (k == 0) R11 = nx;
        if (nx == 0.0 || nx < tol * R11) {
            rank = k;
            if (cr == own && tid == 0) pos[wsl] = -1;   // not kept after all
            break;
        }
        const double sc = s_h[2], tk = s_h[3], g = s_h[4];
        if (cr == 0 && tid == 0) tau[B.coff + k] = tk;
        if (cr == own) { pend_slot = wsl; pend_k = k; pend_beta = s_h[1]; pend_sc = sc; }
        // 5. update own trailing columns, two per warp at a time; squared-norm
        //    downdate (exact recompute when flagged); the warp's best candidate
        const int nl = s_nlive;
        const bool hi = lane >= 16;
        bk = -1;
        bo = INT_MAX;
        for (int t = 2 * warp; t < nl; t += 2 * kQW) {
            const int l1 = lives[t];
            const bool h2 = t + 1 < nl;
            const int l2 = h2 ? lives[t + 1] : l1;
            double *a1 = A + (size_t)l1 * ld_loc;
            double *a2 = A + (size_t)l2 * ld_loc;
            double p1 = 0.0, p2 = 0.0;
            for (int i = k + 1 + lane; i < m; i += 32) {
                const double x = vb[i];
                p1 = fma(x, a1[i], p1);
                p2 = fma(x, a2[i], p2);
            }
            // lanes 0-15 end with column 1's dot product, lanes 16-31 with column 2's
            double dot = (hi ? p2 : p1) + __shfl_xor_sync(kFull, hi ? p1 : p2, 16);
            for (int o = 8; o; o >>= 1) dot += __shfl_xor_sync(kFull, dot, o);
            const int lo = hi ? l2 : l1;
            double *ao = hi ? a2 : a1;
            const double akc = ao[k];
            const double d = fma(g, dot, tk * akc);
            const double e = d * sc;
            const double rkc = akc - d;
            const double e1 = __shfl_sync(kFull, e, 0), e2 = __shfl_sync(kFull, e, 16);
            for (int i = k + 1 + lane; i < m; i += 32) {
                const double x = vb[i];
                a1[i] = fma(-e1, x, a1[i]);
                if (h2) a2[i] = fma(-e2, x, a2[i]);
            }
            double c2;
            const bool again = downdate(cn2[lo], thr[lo], rkc, &c2);
            const bool ag1 = __shfl_sync(kFull, again, 0), ag2 = h2 && __shfl_sync(kFull, again, 16);
            if (ag1 || ag2) {
                double q1 = 0.0, q2 = 0.0;
                for (int i = k + 1 + lane; i < m; i += 32) {
                    q1 = fma(a1[i], a1[i], q1);
                    q2 = fma(a2[i], a2[i], q2);
                }
                double q = (hi ? q2 : q1) + __shfl_xor_sync(kFull, hi ? q1 : q2, 16);
                for (int o = 8; o; o >>= 1) q += __shfl_xor_sync(kFull, q, o);
                if (again) c2 = q;
            }
            __syncwarp();
            if ((lane & 15) == 0 && (!hi || h2)) {
                ao[k] = rkc;
                cn2[lo] = c2;
                if (again) thr[lo] = tol3z * c2;
            }
            const double c21 = __shfl_sync(kFull, c2, 0), c22 = __shfl_sync(kFull, c2, 16);
            const int o1 = cr + C * l1, o2 = cr + C * l2;
            if (key_better(norm_key(c21), o1, bk, bo)) { bk = norm_key(c21); bo = o1; }
            if (h2 && key_better(norm_key(c22), o2, bk, bo)) { bk = norm_key(c22); bo = o2; }
        }
        push(par ^ 1, bk, bo);
    }
    // every CTA has finished reading pivot columns; finish the last deferred write
    cl.sync();
    if (pend_slot >= 0) {
        const double *vp = (pend_k & 1) ? vbuf2 : vbuf;
        double *x = A + (size_t)pend_slot * ld_loc;
        for (int i = pend_k + 1 + tid; i < m; i += kQT) x[i] = vp[i] * pend_sc;
        if (tid == 0) x[pend_k] = pend_beta;
    }
    __syncthreads();
    // positions of the dropped columns: rank + (dropped columns of lower CTAs) + local order
    if (tid == 0) {
        int nd = 0;
        for (int l = 0; l < nloc; ++l) nd += pos[l] < 0;
        s_ndrop = nd;
    }
    cl.sync();
    if (tid == 0) {
        int base = rank;
        for (int r = 0; r < cr; ++r) base += *cl.map_shared_rank(&s_ndrop, r);
        for (int l = 0; l < nloc; ++l)
            if (pos[l] < 0) pos[l] = base++;
    }
    __syncthreads();
    for (int l = warp; l < nloc; l += kQW) {
        const int p = pos[l];
        for (int i = lane; i < m; i += 32) Wb[(int64_t)p * ld + i] = A[(size_t)l * ld_loc + i];
    }
    for (int l = tid; l < nloc; l += kQT) perm_out[B.coff + pos[l]] = cr + C * l;
    if (cr == 0 && tid == 0) {
        rank_out[b] = rank;
        r11_out[b] = R11;
    }
    cl.sync();   // reflectors in global memory; no DSMEM access after this point
    if (!Qout && !Q32) return;
    // Q_hat = H_0 ... H_{r-1} [I_r; 0], owned columns c < r (c mod C == cr)
    const int r = rank;
    const int nq = (r - cr + C - 1) / C > 0 ? (r - cr + C - 1) / C : 0;
    for (int l = warp; l < nq; l += kQW) {
        const int c = cr + C * l;
        for (int i = lane; i < m; i += 32) A[(size_t)l * ld_loc + i] = (i == c) ? 1.0 : 0.0;
    }
    double *cur = vbuf, *nxt = vbuf2;
    if (r > 0) {
        const double *v = Wb + (int64_t)(r - 1) * ld;
        for (int i = r + tid; i < m; i += kQT) cur[i] = v[i];
    }
    __syncthreads();
    for (int k = r - 1; k >= 0; --k) {
        // prefetch reflector k-1 into registers while reflector k is applied
        double pre[4];
        if (k > 0) {
            const double *v = Wb + (int64_t)(k - 1) * ld;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = k + tid + kQT * j;
                pre[j] = i < m ? v[i] : 0.0;
            }
        }
        const double tk = tau[B.coff + k];
        const int lq = (k - cr + C - 1) / C > 0 ? (k - cr + C - 1) / C : 0;
        for (int l = lq + warp; l < nq; l += kQW) {
            double *q = A + (size_t)l * ld_loc;
            double d = 0.0;
            for (int i = k + 1 + lane; i < m; i += 32) d = fma(cur[i], q[i], d);
            for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            const double qk = q[k];
            d = tk * (qk + d);
            for (int i = k + 1 + lane; i < m; i += 32) q[i] = fma(-d, cur[i], q[i]);
            __syncwarp();
            if (lane == 0) q[k] = qk - d;
        }
        if (k > 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = k + tid + kQT * j;
                if (i < m) nxt[i] = pre[j];
            }
            const double *v = Wb + (int64_t)(k - 1) * ld;   // rows beyond the register prefetch
            for (int i = k + tid + 4 * kQT; i < m; i += kQT) nxt[i] = v[i];
        }
        __syncthreads();
        double *t = cur; cur = nxt; nxt = t;
    }
    for (int l = warp; l < nq; l += kQW) {
        const int c = cr + C * l;
        for (int i = lane; i < ld; i += 32) {     // rows m..ld-1 are padding: zeros
            const double qv = i < m ? A[(size_t)l * ld_loc + i] : 0.0;
            if (Q32) Q32[B.moff + (int64_t)c * ld + i] = (float)qv;
            else Qout[B.moff + (int64_t)c * ld + i] = qv;
        }
    }
}

// ---------------------------------------------------------------------------
// Double-float variant of the cluster kernel, for blocks assembled in FP32
// (their entries are exact double-floats with a zero low word).  Same
// algorithm, data distribution and step structure; the block, the pivot
// column and the trailing squared norms are double-float pairs in shared
// memory, and every per-element operation (dot products, column updates,
// squared norms) and the per-column scalars run on the FP32 pipe.  The
// reflector scalars of a step (norm, beta, tau) are formed once in FP64 from
// the double-float sums.  Pivots compare the high words of the squared
// norms.  The factorisation leaves R and the reflectors in W (FP64) and, for
// Q_hat, double-float copies of the reflectors in the scratch arena Vdf, from
// which Q_hat = H_0 ... H_{r-1} [I_r; 0] is accumulated backwards in
// double-float and rounded to FP32.
// ---------------------------------------------------------------------------
constexpr int kDT = 512;          // threads of a double-float cluster-QR CTA (its FP32 dependency chains want more warps)
constexpr int kDW = kDT / 32;

// An input entry as a double-float: FP32 entries exactly, FP64 entries split
// into their nearest FP32 number and the FP32 rounding of the remainder.
__device__ inline float2 df_in(float x) { return make_float2(x, 0.f); }
__device__ inline float2 df_in(double x) { return df_from_double(x); }

template <typename TM, int C>
__global__ void __launch_bounds__(kDT) k_qrcp_cluster_df(const BlkRec *__restrict__ blks,
                                                         const int32_t *__restrict__ order, const TM *__restrict__ M,
                                                         double *__restrict__ W, double *__restrict__ tau,
                                                         int32_t *__restrict__ perm_out, int32_t *__restrict__ rank_out,
                                                         double *__restrict__ r11_out, double tol, int nloc_max,
                                                         int ld_loc, int k_max, float2 *__restrict__ Vdf,
                                                         float *__restrict__ Q32) {
    cg::cluster_group cl = cg::this_cluster();
    const int cr = (int)cl.block_rank();
    const int b = order ? order[blockIdx.x / C] : (int)(blockIdx.x / C);
    const BlkRec B = blks[b];
    const int m = B.m, K = B.K, ld = B.ldm;
    extern __shared__ __align__(16) float2 smf[];
    float2 *A = smf;                                        // nloc_max x ld_loc
    float2 *vbuf = A + (size_t)nloc_max * ld_loc;           // ld_loc: pivot column of even steps (later: Q prefetch)
    float2 *vbuf2 = vbuf + ld_loc;                          // ld_loc: pivot column of odd steps
    float2 *taud = vbuf2 + ld_loc;                          // k_max: tau of every step
    float2 *cn2 = taud + k_max;                             // nloc_max: squared trailing norms
    float *thr = reinterpret_cast<float *>(cn2 + nloc_max);  // nloc_max: tol3z * last exact squared norm
    int *pos = reinterpret_cast<int *>(thr + nloc_max);     // nloc_max: position, -1 while trailing
    int *lives = pos + nloc_max;                            // nloc_max: slots of the trailing columns
    int *where = lives + nloc_max;                          // nloc_max: index of a slot in lives
    __shared__ Cand cands[2][C * kDW];
    __shared__ float2 s_red[kDW];
    __shared__ double s_nx, s_tau;
    __shared__ float2 s_h[3];    // beta, sc, g of the step (tau goes to taud)
    __shared__ int s_ndrop;
    __shared__ int s_nlive;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nloc = (K - cr + C - 1) / C;
    double *Wb = W + B.moff;
    const float tol3z = 1.4901161193847656e-08f;   // sqrt of the FP64 epsilon, as in the FP64 kernels
    // pivot key of a normalised squared norm (h >= 0): the high word's bits,
    // then the low word's bits mapped to an order-preserving unsigned
    auto fkey = [](float2 c2) {
        unsigned lo = __float_as_uint(c2.y);
        lo = (lo & 0x80000000u) ? ~lo : (lo | 0x80000000u);
        return ((long long)__float_as_int(c2.x) << 32) | (long long)lo;
    };

    auto push = [&](int par, long long key, int orig) {
        if (lane < C) {
            Cand *dst = cl.map_shared_rank(&cands[par][cr * kDW + warp], lane);
            *reinterpret_cast<longlong2 *>(dst) = make_longlong2(key, (long long)orig);
        }
    };
    cl.sync();

    long long bk = -1;
    int bo = INT_MAX;
    for (int l = warp; l < nloc; l += kDW) {
        const int c = cr + C * l;
        const TM *src = M + B.moff + (int64_t)c * ld;
        float sh = 0.f, sl = 0.f;
        for (int i = lane; i < m; i += 32) {
            const float2 a = df_in(src[i]);
            A[(size_t)l * ld_loc + i] = a;
            df_acc(a, a, sh, sl);
        }
        float2 s2 = make_float2(sh, sl);
        for (int o = 16; o; o >>= 1) s2 = df_xor_add(s2, o);
        if (lane == 0) {
            cn2[l] = s2;
            thr[l] = tol3z * s2.x;
            pos[l] = -1;
            lives[l] = l;
            where[l] = l;
        }
        if (key_better(fkey(s2), c, bk, bo)) { bk = fkey(s2); bo = c; }
    }
    if (tid == 0) s_nlive = nloc;
    push(0, bk, bo);
    const int steps = m < K ? m : K;
    double R11 = 0.0;
    int rank = steps;
    int pend_slot = -1, pend_k = 0;
    float2 pend_beta = make_float2(0.f, 0.f), pend_sc = make_float2(0.f, 0.f);
    for (int k = 0; k < steps; ++k) {
        const int par = k & 1;
        float2 *vb = par ? vbuf2 : vbuf;
        cl.sync();
        // 1. winner over the cluster, in every warp
        {
            bk = -1;
            bo = INT_MAX;
            for (int t = lane; t < C * kDW; t += 32) {
                const longlong2 cd = *reinterpret_cast<const longlong2 *>(&cands[par][t]);
                if (key_better(cd.x, (int)cd.y, bk, bo)) { bk = cd.x; bo = (int)cd.y; }
            }
            for (int o = 16; o; o >>= 1) {
                const long long k2 = __shfl_xor_sync(kFull, bk, o);
                const int o2 = __shfl_xor_sync(kFull, bo, o);
                if (key_better(k2, o2, bk, bo)) { bk = k2; bo = o2; }
            }
        }
        const int own = bo % C, wsl = bo / C;
        // 2. deferred write of the previous reflector (v = x sc, beta on the diagonal)
        if (pend_slot >= 0) {
            const float2 *vp = par ? vbuf : vbuf2;
            float2 *x = A + (size_t)pend_slot * ld_loc;
            for (int i = pend_k + 1 + tid; i < m; i += kDT) x[i] = df_mul(vp[i], pend_sc);
            if (tid == 0) x[pend_k] = pend_beta;
            pend_slot = -1;
        }
        if (cr == own && tid == 0) {
            pos[wsl] = k;
            const int at = where[wsl], last = lives[s_nlive - 1];
            lives[at] = last;
            where[last] = at;
            s_nlive -= 1;
        }
        // 3. copy the pivot column (rows k..m) from its owner, sum of squares
        {
            const float2 *rx = cl.map_shared_rank(A, own) + (size_t)wsl * ld_loc;
            float sh = 0.f, sl = 0.f;
            for (int i = k + tid; i < m; i += kDT) {
                const float2 x = rx[i];
                vb[i] = x;
                df_acc(x, x, sh, sl);
            }
            float2 s2 = make_float2(sh, sl);
            for (int o = 16; o; o >>= 1) s2 = df_xor_add(s2, o);
            if (lane == 0) s_red[warp] = s2;
        }
        __syncthreads();
        // 4. exact norm and reflector scalars (one warp), in double-float:
        //    beta = -sign(alpha) nx, sc = 1 / (alpha - beta), g = -1 / beta,
        //    tau = (alpha - beta) g, from one reciprocal (as house_scalars)
        if (warp == 0) {
            float2 t = lane < kDW ? s_red[lane] : make_float2(0.f, 0.f);
            for (int o = kDW / 2; o; o >>= 1) t = df_xor_add(t, o);
            if (lane == 0) {
                const float2 nxd = t.x > 0.f ? df_sqrt(t) : make_float2(0.f, 0.f);
                s_nx = df_to_double(nxd);
                if (nxd.x > 0.f) {
                    const float2 alpha = vb[k];
                    const float2 beta = alpha.x >= 0.f ? df_neg(nxd) : nxd;
                    const float2 amb = df_sub(alpha, beta);
                    const float2 inv = df_rcp(df_mul(amb, beta));
                    const float2 g = df_neg(df_mul(amb, inv));
                    const float2 tk = df_mul(amb, g);
                    s_h[0] = beta;
                    s_h[1] = df_mul(beta, inv);
                    s_h[2] = g;
                    taud[k] = tk;
                    s_tau = df_to_double(tk);
                }
            }
        }
        __syncthreads();
        const double nx = s_nx;
        if (k == 0) R11 = nx;
        if (nx == 0.0 || nx < tol * R11) {
            rank = k;
            if (cr == own && tid == 0) pos[wsl] = -1;
            break;
        }
        const float2 sc = s_h[1], tk = taud[k], g = s_h[2];
        if (cr == 0 && tid == 0) tau[B.coff + k] = s_tau;
        if (cr == own) { pend_slot = wsl; pend_k = k; pend_beta = s_h[0]; pend_sc = sc; }
        // 5. update own trailing columns, two per warp at a time
        const int nl = s_nlive;
        const bool hi = lane >= 16;
        bk = -1;
        bo = INT_MAX;
        for (int t = 2 * warp; t < nl; t += 2 * kDW) {
            const int l1 = lives[t];
            const bool h2 = t + 1 < nl;
            const int l2 = h2 ? lives[t + 1] : l1;
            float2 *a1 = A + (size_t)l1 * ld_loc;
            float2 *a2 = A + (size_t)l2 * ld_loc;
            float p1h = 0.f, p1l = 0.f, p2h = 0.f, p2l = 0.f;
            for (int i = k + 1 + lane; i < m; i += 32) {
                const float2 x = vb[i];
                df_acc(x, a1[i], p1h, p1l);
                df_acc(x, a2[i], p2h, p2l);
            }
            // lanes 0-15 end with column 1's dot product, lanes 16-31 with column 2's
            const float2 keep = hi ? make_float2(p2h, p2l) : make_float2(p1h, p1l);
            const float2 send = hi ? make_float2(p1h, p1l) : make_float2(p2h, p2l);
            float2 dot = df_add(keep, make_float2(__shfl_xor_sync(kFull, send.x, 16), __shfl_xor_sync(kFull, send.y, 16)));
            for (int o = 8; o; o >>= 1) dot = df_xor_add(dot, o);
            const int lo = hi ? l2 : l1;
            float2 *ao = hi ? a2 : a1;
            const float2 akc = ao[k];
            const float2 d = df_add(df_mul(g, dot), df_mul(tk, akc));
            const float2 e = df_mul(d, sc);
            const float2 rkc = df_sub(akc, d);
            const float2 e1 = make_float2(__shfl_sync(kFull, e.x, 0), __shfl_sync(kFull, e.y, 0));
            const float2 e2 = make_float2(__shfl_sync(kFull, e.x, 16), __shfl_sync(kFull, e.y, 16));
            for (int i = k + 1 + lane; i < m; i += 32) {
                const float2 x = vb[i];
                a1[i] = df_axmy(a1[i], e1, x);
                if (h2) a2[i] = df_axmy(a2[i], e2, x);
            }
            const float2 c2o = cn2[lo];
            float2 c2 = make_float2(0.f, 0.f);
            bool again = false;
            if (c2o.x != 0.f) {
                c2 = df_sub(c2o, df_mul(rkc, rkc));
                again = !(c2.x > thr[lo]);
            }
            const bool ag1 = __shfl_sync(kFull, again, 0), ag2 = h2 && __shfl_sync(kFull, again, 16);
            if (ag1 || ag2) {
                float q1h = 0.f, q1l = 0.f, q2h = 0.f, q2l = 0.f;
                for (int i = k + 1 + lane; i < m; i += 32) {
                    const float2 u1 = a1[i], u2 = a2[i];
                    df_acc(u1, u1, q1h, q1l);
                    df_acc(u2, u2, q2h, q2l);
                }
                const float2 qk = hi ? make_float2(q2h, q2l) : make_float2(q1h, q1l);
                const float2 qs = hi ? make_float2(q1h, q1l) : make_float2(q2h, q2l);
                float2 q = df_add(qk, make_float2(__shfl_xor_sync(kFull, qs.x, 16), __shfl_xor_sync(kFull, qs.y, 16)));
                for (int o = 8; o; o >>= 1) q = df_xor_add(q, o);
                if (again) c2 = q;
            }
            __syncwarp();
            if ((lane & 15) == 0 && (!hi || h2)) {
                ao[k] = rkc;
                cn2[lo] = c2;
                if (again) thr[lo] = tol3z * c2.x;
            }
            const long long k1 = fkey(make_float2(__shfl_sync(kFull, c2.x, 0), __shfl_sync(kFull, c2.y, 0)));
            const long long k2 = fkey(make_float2(__shfl_sync(kFull, c2.x, 16), __shfl_sync(kFull, c2.y, 16)));
            const int o1 = cr + C * l1, o2 = cr + C * l2;
            if (key_better(k1, o1, bk, bo)) { bk = k1; bo = o1; }
            if (h2 && key_better(k2, o2, bk, bo)) { bk = k2; bo = o2; }
        }
        push(par ^ 1, bk, bo);
    }
    cl.sync();
    if (pend_slot >= 0) {
        const float2 *vp = (pend_k & 1) ? vbuf2 : vbuf;
        float2 *x = A + (size_t)pend_slot * ld_loc;
        for (int i = pend_k + 1 + tid; i < m; i += kDT) x[i] = df_mul(vp[i], pend_sc);
        if (tid == 0) x[pend_k] = pend_beta;
    }
    __syncthreads();
    // positions of the dropped columns: rank + (dropped columns of lower CTAs) + local order
    if (tid == 0) {
        int nd = 0;
        for (int l = 0; l < nloc; ++l) nd += pos[l] < 0;
        s_ndrop = nd;
    }
    cl.sync();
    if (tid == 0) {
        int base = rank;
        for (int r = 0; r < cr; ++r) base += *cl.map_shared_rank(&s_ndrop, r);
        for (int l = 0; l < nloc; ++l)
            if (pos[l] < 0) pos[l] = base++;
    }
    __syncthreads();
    for (int l = warp; l < nloc; l += kDW) {
        const int p = pos[l];
        const float2 *src = A + (size_t)l * ld_loc;
        for (int i = lane; i < m; i += 32) Wb[(int64_t)p * ld + i] = df_to_double(src[i]);
        if (Vdf && p < rank)
            for (int i = lane; i < m; i += 32) Vdf[B.moff + (int64_t)p * ld + i] = src[i];
    }
    for (int l = tid; l < nloc; l += kDT) perm_out[B.coff + pos[l]] = cr + C * l;
    if (cr == 0 && tid == 0) {
        rank_out[b] = rank;
        r11_out[b] = R11;
    }
    cl.sync();   // reflectors in global memory; no DSMEM access after this point
    if (!Q32 || !Vdf) return;
    // Q_hat = H_0 ... H_{r-1} [I_r; 0], owned columns c < r (c mod C == cr),
    // two columns per warp at a time
    const int r = rank;
    const int nq = (r - cr + C - 1) / C > 0 ? (r - cr + C - 1) / C : 0;
    for (int l = warp; l < nq; l += kDW) {
        const int c = cr + C * l;
        for (int i = lane; i < m; i += 32) A[(size_t)l * ld_loc + i] = make_float2(i == c ? 1.f : 0.f, 0.f);
    }
    const float2 *Vb = Vdf + B.moff;
    float2 *cur = vbuf, *nxt = vbuf2;
    if (r > 0)
        for (int i = r + tid; i < m; i += kDT) cur[i] = Vb[(int64_t)(r - 1) * ld + i];
    __syncthreads();
    const bool hi = lane >= 16;
    for (int k = r - 1; k >= 0; --k) {
        float2 pre[4];
        if (k > 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = k + tid + kDT * j;
                pre[j] = i < m ? Vb[(int64_t)(k - 1) * ld + i] : make_float2(0.f, 0.f);
            }
        }
        const float2 tk = taud[k];
        const int lq = (k - cr + C - 1) / C > 0 ? (k - cr + C - 1) / C : 0;
        for (int t = lq + 2 * warp; t < nq; t += 2 * kDW) {
            const bool h2 = t + 1 < nq;
            float2 *q1 = A + (size_t)t * ld_loc;
            float2 *q2 = A + (size_t)(h2 ? t + 1 : t) * ld_loc;
            float p1h = 0.f, p1l = 0.f, p2h = 0.f, p2l = 0.f;
            for (int i = k + 1 + lane; i < m; i += 32) {
                const float2 v = cur[i];
                df_acc(v, q1[i], p1h, p1l);
                df_acc(v, q2[i], p2h, p2l);
            }
            const float2 keep = hi ? make_float2(p2h, p2l) : make_float2(p1h, p1l);
            const float2 send = hi ? make_float2(p1h, p1l) : make_float2(p2h, p2l);
            float2 dot = df_add(keep, make_float2(__shfl_xor_sync(kFull, send.x, 16), __shfl_xor_sync(kFull, send.y, 16)));
            for (int o = 8; o; o >>= 1) dot = df_xor_add(dot, o);
            float2 *qo = hi ? q2 : q1;
            const float2 qk = qo[k];
            const float2 d = df_mul(tk, df_add(qk, dot));
            const float2 d1 = make_float2(__shfl_sync(kFull, d.x, 0), __shfl_sync(kFull, d.y, 0));
            const float2 d2 = make_float2(__shfl_sync(kFull, d.x, 16), __shfl_sync(kFull, d.y, 16));
            for (int i = k + 1 + lane; i < m; i += 32) {
                const float2 v = cur[i];
                q1[i] = df_axmy(q1[i], d1, v);
                if (h2) q2[i] = df_axmy(q2[i], d2, v);
            }
            __syncwarp();
            if ((lane & 15) == 0 && (!hi || h2)) qo[k] = df_sub(qk, d);
        }
        if (k > 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = k + tid + kDT * j;
                if (i < m) nxt[i] = pre[j];
            }
            for (int i = k + tid + 4 * kDT; i < m; i += kDT) nxt[i] = Vb[(int64_t)(k - 1) * ld + i];
        }
        __syncthreads();
        float2 *tt = cur; cur = nxt; nxt = tt;
    }
    for (int l = warp; l < nq; l += kDW) {
        const int c = cr + C * l;
        for (int i = lane; i < ld; i += 32)
            Q32[B.moff + (int64_t)c * ld + i] = i < m ? df_to_float(A[(size_t)l * ld_loc + i]) : 0.f;
    }
}

template <typename TM, int C>
static rfm_status launch_cluster(const FilterBufs &F, double tol, int nloc, int ldl, size_t smem, cudaStream_t st) {
    auto kern = k_qrcp_cluster<TM, C>;
    RFM_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (C > 8) RFM_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(F.n_blocks * C));
    cfg.blockDim = dim3(kQT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    RFM_CUDA_CHECK(cudaLaunchKernelEx(&cfg, kern, F.blk, F.order, (const TM *)F.M, F.W, F.tau, F.perm, F.rank, F.r11, tol,
                                      nloc, ldl, F.Q64, F.Q32));
    return RFM_OK;
}

// Shared-memory bytes of the cluster kernel for cluster size C (the
// double-float kernel adds the tau of every step).
static size_t cluster_smem(int64_t max_m, int64_t max_K, int C, int *nloc, int *ldl, bool df = false) {
    *ldl = (int)((max_m + 1) / 2 * 2);
    *nloc = (int)((max_K + C - 1) / C);
    return ((size_t)(*nloc) * (*ldl) + 2 * (size_t)(*ldl) + (df ? (size_t)max_K : 0)) * 8 + (size_t)(*nloc) * 32 + 64;
}

// FP32-assembled blocks go to the double-float kernel unless Q_hat is wanted
// in FP64 (RFM_OPT_QR_DOUBLE_FLOAT = 0 keeps them on the FP64 kernel).  Its
// Q_hat path keeps double-float copies of the reflectors in the FP64
// operator arena, which the FP32 operator leaves free.
// With RFM_OPT_QR_DOUBLE_FLOAT = 2, FP64 blocks whose Q_hat is wanted in FP32
// take it too (their entries split into double-floats on load).
static int g_qr_df = 1;
static bool use_df(const FilterBufs &F, int elem) {
    const bool kind = (elem == 4 && g_qr_df) || (elem == 8 && g_qr_df == 2 && F.Q32 != nullptr);
    return kind && F.Q64 == nullptr && (F.Q32 == nullptr || F.Op != nullptr);
}

template <typename TM, int C>
static rfm_status launch_cluster_df(const FilterBufs &F, double tol, int nloc, int ldl, size_t smem,
                                    cudaStream_t st) {
    auto kern = k_qrcp_cluster_df<TM, C>;
    RFM_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (C > 8) RFM_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(F.n_blocks * C));
    cfg.blockDim = dim3(kDT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    float2 *vdf = F.Q32 ? reinterpret_cast<float2 *>(F.Op) : nullptr;
    RFM_CUDA_CHECK(cudaLaunchKernelEx(&cfg, kern, F.blk, F.order, (const TM *)F.M, F.W, F.tau, F.perm, F.rank, F.r11,
                                      tol, nloc, ldl, (int)F.max_K, vdf, F.Q32));
    return RFM_OK;
}

template <typename TM>
static rfm_status launch_cluster_c(int C, const FilterBufs &F, double tol, cudaStream_t st) {
    int nloc = 0, ldl = 0;
    if (use_df(F, (int)sizeof(TM))) {
        const size_t smem = cluster_smem(F.max_m, F.max_K, C, &nloc, &ldl, true);
        switch (C) {
            case 1: return launch_cluster_df<TM, 1>(F, tol, nloc, ldl, smem, st);
            case 2: return launch_cluster_df<TM, 2>(F, tol, nloc, ldl, smem, st);
            case 4: return launch_cluster_df<TM, 4>(F, tol, nloc, ldl, smem, st);
            case 8: return launch_cluster_df<TM, 8>(F, tol, nloc, ldl, smem, st);
            default: return launch_cluster_df<TM, 16>(F, tol, nloc, ldl, smem, st);
        }
    }
    const size_t smem = cluster_smem(F.max_m, F.max_K, C, &nloc, &ldl);
    switch (C) {
        case 1: return launch_cluster<TM, 1>(F, tol, nloc, ldl, smem, st);
        case 2: return launch_cluster<TM, 2>(F, tol, nloc, ldl, smem, st);
        case 4: return launch_cluster<TM, 4>(F, tol, nloc, ldl, smem, st);
        case 8: return launch_cluster<TM, 8>(F, tol, nloc, ldl, smem, st);
        default: return launch_cluster<TM, 16>(F, tol, nloc, ldl, smem, st);
    }
}

// Cluster-size autotuner: per block shape (largest block rows and features,
// input precision, block count) the fastest feasible cluster size, timed
// with events on the caller's stream (after one untimed launch of the same
// size) and remembered for the process.
// Every cluster size computes the same factors (per-column arithmetic and
// pivot ties do not depend on how columns are spread over CTAs), so the last
// timed run leaves a valid result.
static int g_autotune = 0;
static int g_qr_warps = 32;  // warps per CTA of the global-memory QR kernels
void set_qr_warps(int v) { g_qr_warps = v; }
static int g_qr_panel = 8;   // panel width of the double-float global QR and Q_hat formation (1, 2, 4 or 8)
void set_qr_panel(int v) { g_qr_panel = v; }
struct TuneEntry {
    int64_t max_m, max_K, n_blocks;
    int elem, C;
};
static std::mutex g_tune_mu;
static std::vector<TuneEntry> g_tune;

// kernel family of a launch: 2 = double-float, 4 / 8 = FP64 arithmetic on FP32 / FP64 blocks
static int tune_kind(const FilterBufs &F, int elem) { return use_df(F, elem) ? 2 : elem; }

static int cached_cluster(const FilterBufs &F, int elem) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const TuneEntry &e : g_tune)
        if (e.max_m == F.max_m && e.max_K == F.max_K && e.n_blocks == F.n_blocks && e.elem == tune_kind(F, elem))
            return e.C;
    return 0;
}

template <typename TM>
static rfm_status autotune_cluster(const FilterBufs &F, double tol, int C_min, cudaStream_t st, int *best) {
    cudaEvent_t e0, e1;
    RFM_CUDA_CHECK(cudaEventCreate(&e0));
    RFM_CUDA_CHECK(cudaEventCreate(&e1));
    float best_ms = 0.f;
    *best = C_min;
    rfm_status rc = RFM_OK;
    for (int C = C_min; C <= 16; C *= 2) {
        // 16 CTAs per cluster is a non-portable size: ask whether this device
        // can place such clusters before timing it
        if (C > 8) {
            int nclusters = 0;
            int nloc = 0, ldl = 0;
            const bool dfk = use_df(F, (int)sizeof(TM));
            const size_t smem = cluster_smem(F.max_m, F.max_K, C, &nloc, &ldl, dfk);
            const void *kern = dfk ? (const void *)k_qrcp_cluster_df<TM, 16> : (const void *)k_qrcp_cluster<TM, 16>;
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
                cudaGetLastError();
                break;
            }
            cudaLaunchConfig_t q = {};
            q.gridDim = dim3(16);
            q.blockDim = dim3(dfk ? kDT : kQT);
            q.dynamicSmemBytes = smem;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = 16;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            q.attrs = at;
            q.numAttrs = 1;
            if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &q) != cudaSuccess || nclusters < 1) {
                cudaGetLastError();
                break;
            }
        }
        // one untimed launch first: a kernel's first launch in a process also
        // loads its module
        rc = launch_cluster_c<TM>(C, F, tol, st);
        cudaEventRecord(e0, st);
        if (rc == RFM_OK) rc = launch_cluster_c<TM>(C, F, tol, st);
        cudaEventRecord(e1, st);
        if (rc != RFM_OK) {
            if (C > 8 && C > C_min) {   // an optional size the device refused: the earlier runs' result stands
                cudaGetLastError();
                rc = RFM_OK;
            }
            break;
        }
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            set_error("QR autotuner: timing run failed");
            rc = RFM_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (C == C_min || ms < best_ms) {
            best_ms = ms;
            *best = C;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != RFM_OK) return rc;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.push_back(TuneEntry{F.max_m, F.max_K, F.n_blocks, tune_kind(F, (int)sizeof(TM)), *best});
    return RFM_OK;
}

// Warps-per-block tuner of the global-memory kernels (same shape key as the
// cluster tuner, their own table); the candidates run in the order 8, 16, 32.
static std::vector<TuneEntry> g_tune_global;

static int cached_global(const FilterBufs &F, int kind) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const TuneEntry &e : g_tune_global)
        if (e.max_m == F.max_m && e.max_K == F.max_K && e.n_blocks == F.n_blocks && e.elem == kind) return e.C;
    return 0;
}

template <typename Run>
static rfm_status autotune_global(const FilterBufs &F, int kind, cudaStream_t st, Run run, int *best) {
    cudaEvent_t e0, e1;
    RFM_CUDA_CHECK(cudaEventCreate(&e0));
    RFM_CUDA_CHECK(cudaEventCreate(&e1));
    float best_ms = 0.f;
    *best = 32;
    rfm_status rc = RFM_OK;
    for (int nw : {8, 16, 32}) {
        cudaEventRecord(e0, st);
        rc = run(nw);
        cudaEventRecord(e1, st);
        if (rc != RFM_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            set_error("QR autotuner: timing run failed");
            rc = RFM_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (nw == 8 || ms < best_ms) {
            best_ms = ms;
            *best = nw;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != RFM_OK) return rc;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_global.push_back(TuneEntry{F.max_m, F.max_K, F.n_blocks, kind, *best});
    return RFM_OK;
}

// Panel-width tuner of the double-float global kernels (QR and Q_hat
// formation): times each candidate once, keeps the fastest for the process
// and leaves its factors (the candidate last timed is re-run when it is not
// the fastest).
template <typename Run>
static rfm_status autotune_panel(const FilterBufs &F, int kind, cudaStream_t st, Run run, const std::vector<int> &cands,
                                 int *best) {
    cudaEvent_t e0, e1;
    RFM_CUDA_CHECK(cudaEventCreate(&e0));
    RFM_CUDA_CHECK(cudaEventCreate(&e1));
    float best_ms = 0.f;
    rfm_status rc = RFM_OK;
    for (size_t k = 0; k < cands.size(); ++k) {
        cudaEventRecord(e0, st);
        rc = run(cands[k]);
        cudaEventRecord(e1, st);
        if (rc != RFM_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            set_error("QR autotuner: timing run failed");
            rc = RFM_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (k == 0 || ms < best_ms) {
            best_ms = ms;
            *best = cands[k];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == RFM_OK && !cands.empty() && *best != cands.back()) rc = run(*best);
    if (rc != RFM_OK) return rc;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_global.push_back(TuneEntry{F.max_m, F.max_K, F.n_blocks, kind, *best});
    return RFM_OK;
}

template <typename TM>
static rfm_status launch_filter_t(const FilterBufs &F, double tol, cudaStream_t st) {
    const unsigned nb = (unsigned)F.n_blocks;
    const size_t kSmemCap = 220 * 1024;
    int C = 0, nloc = 0, ldl = 0;
    size_t smem = 0;
    const bool dfk = use_df(F, (int)sizeof(TM));
    for (int c : {1, 2, 4, 8}) {
        if (F.no_cluster) break;
        smem = cluster_smem(F.max_m, F.max_K, c, &nloc, &ldl, dfk);
        if (smem <= kSmemCap) { C = c; break; }
    }
    if (C > 0) {
        ProfScope ps(F.fit ? "k_qrcp_cluster_fit" : "k_qrcp_cluster", st);
        rfm_status rc;
        int tuned = g_autotune ? cached_cluster(F, (int)sizeof(TM)) : 0;
        if (g_autotune && tuned == 0) {
            rc = autotune_cluster<TM>(F, tol, C, st, &tuned);   // leaves a valid result
        } else {
            rc = launch_cluster_c<TM>(tuned ? tuned : C, F, tol, st);
        }
        if (rc != RFM_OK) return rc;
    } else {
        const size_t sm = (size_t)F.max_K * (2 * sizeof(double) + sizeof(int));
        // FP32-assembled blocks in double-float (RFM_OPT_QR_DOUBLE_FLOAT, as the cluster kernels)
        const bool gdf = sizeof(TM) == 4 && g_qr_df != 0 && !F.fit &&
                         sizeof(float2) * (size_t)F.max_m + (size_t)F.max_K * 16 <= 200 * 1024;
        // Q_hat of the double-float path: panel width pw (1 = one reflector
        // per pass; 2, 4, 8 = compact WY panels in shared memory)
        const size_t ldmax = (size_t)((F.max_m + kLdAlign - 1) / kLdAlign * kLdAlign);
        auto panel_fits = [&](int pw) { return pw == 1 || sizeof(float2) * (size_t)pw * ldmax <= 200 * 1024; };
        // the panel QR's shared memory: V (pw x ld), F (K x pw), norms, thresholds, permutation
        auto qr_panel_smem = [&](int pw) {
            return sizeof(float2) * ((size_t)pw * ldmax + (size_t)F.max_K * pw + (size_t)F.max_K) +
                   (size_t)F.max_K * (sizeof(float) + sizeof(int));
        };
        // (the QR's panels stop at 4 steps: with 8 its 1024-thread CTAs spill
        // under their 64 registers per thread, 618 against 596 ms on heat)
        auto qr_panel_for = [&](int pw) {
            for (int q : {4, 2})
                if (q <= pw && qr_panel_smem(q) <= 225 * 1024) return q;
            return 1;
        };
        auto form_gdf = [&](auto nwc, int pw) -> rfm_status {
            constexpr int NW = decltype(nwc)::value;
            ProfScope ps(F.fit ? "k_form_q_fit" : "k_form_q", st);
            if (pw == 1) {
                const size_t smq = sizeof(float2) * (size_t)F.max_m;
                RFM_CUDA_CHECK(cudaFuncSetAttribute(k_form_q_gdf<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smq));
                k_form_q_gdf<NW><<<nb, NW * 32, smq, st>>>(F.blk, F.W, F.tau, F.rank, F.Op, F.Q32);
            } else {
                const size_t smq = sizeof(float2) * (size_t)pw * ldmax;
                auto launch = [&](auto kern) -> rfm_status {
                    RFM_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smq));
                    kern<<<nb, NW * 32, smq, st>>>(F.blk, F.W, F.tau, F.rank, F.Op, F.Q32);
                    return RFM_OK;
                };
                const rfm_status lr = pw == 2 ? launch(k_form_q_gdf_blk<NW, 2>)
                                    : pw == 4 ? launch(k_form_q_gdf_blk<NW, 4>) : launch(k_form_q_gdf_blk<NW, 8>);
                if (lr != RFM_OK) return lr;
            }
            RFM_CUDA_CHECK(cudaGetLastError());
            return RFM_OK;
        };
        int panel = 1;
        for (int pw : {8, 4, 2})
            if (pw <= g_qr_panel && panel_fits(pw)) { panel = pw; break; }
        auto global_qr = [&](auto nwc) -> rfm_status {
            constexpr int NW = decltype(nwc)::value;
            if (gdf) {
                // FP32-assembled blocks in double-float arithmetic: one step at
                // a time (the pivot column in shared memory) or in panels of
                // qp steps with the trailing update deferred
                ProfScope ps(F.fit ? "k_qrcp_fit" : "k_qrcp", st);
                const int qp = qr_panel_for(panel);
                if (qp == 1) {
                    const size_t smd = sizeof(float2) * (size_t)F.max_m + (size_t)F.max_K * (sizeof(float2) + sizeof(float) + sizeof(int));
                    RFM_CUDA_CHECK(cudaFuncSetAttribute(k_qrcp_gdf<TM, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smd));
                    k_qrcp_gdf<TM, NW><<<nb, NW * 32, smd, st>>>(F.blk, (const TM *)F.M, F.W, F.tau, F.perm, F.rank, F.r11, tol);
                } else {
                    const size_t smd = qr_panel_smem(qp);
                    auto launch = [&](auto kern) -> rfm_status {
                        RFM_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smd));
                        kern<<<nb, NW * 32, smd, st>>>(F.blk, (const TM *)F.M, F.W, F.tau, F.perm, F.rank, F.r11, tol);
                        return RFM_OK;
                    };
                    const rfm_status lr = qp == 2 ? launch(k_qrcp_gdf_blk<TM, NW, 2>) : launch(k_qrcp_gdf_blk<TM, NW, 4>);
                    if (lr != RFM_OK) return lr;
                }
                RFM_CUDA_CHECK(cudaGetLastError());
            } else {
                ProfScope ps(F.fit ? "k_qrcp_fit" : "k_qrcp", st);
                RFM_CUDA_CHECK(cudaFuncSetAttribute(k_qrcp<TM, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
                k_qrcp<TM, NW><<<nb, NW * 32, sm, st>>>(F.blk, (const TM *)F.M, F.W, F.tau, F.perm, F.rank, F.r11, tol);
                RFM_CUDA_CHECK(cudaGetLastError());
            }
            if (gdf && F.Q32 && !F.Q64) {
                return form_gdf(nwc, panel);
            } else if (F.Q64 || F.Q32) {
                ProfScope ps(F.fit ? "k_form_q_fit" : "k_form_q", st);
                k_form_q<NW><<<nb, NW * 32, 0, st>>>(F.blk, F.W, F.tau, F.rank, F.Op, F.Q32);
                RFM_CUDA_CHECK(cudaGetLastError());
            }
            return RFM_OK;
        };
        // (32 warps, one 1024-thread CTA per block: the heat workload's filter
        // takes 1.87 s against 2.19 s with 8 warps and 2.86 s with 4)
        auto run_warps = [&](int nw) -> rfm_status {
            switch (nw) {
            case 4: return global_qr(std::integral_constant<int, 4>{});
            case 8: return global_qr(std::integral_constant<int, 8>{});
            case 16: return global_qr(std::integral_constant<int, 16>{});
            default: return global_qr(std::integral_constant<int, 32>{});
            }
        };
        const int kind = tune_kind(F, (int)sizeof(TM)) + (gdf ? 16 : 0);
        int nw = g_autotune ? cached_global(F, kind) : g_qr_warps;
        rfm_status rc;
        const bool tune_panel = g_autotune && gdf && F.Q32 && !F.Q64;
        const int pkind = kind + 32;
        if (tune_panel) {
            const int pc = cached_global(F, pkind);
            if (pc > 0) panel = pc;
        }
        if (nw == 0) {
            // autotuner (RFM_OPT_AUTOTUNE): time 8, 16 and 32 warps per block
            // once each for this block shape, keep the fastest for the
            // process, and leave its factors (the variants agree to rounding)
            rc = autotune_global(F, kind, st, run_warps, &nw);
            if (rc == RFM_OK && nw != 32) rc = run_warps(nw);
            if (rc == RFM_OK && tune_panel) {
                // then the panel width of the QR and the Q_hat formation with
                // those warps (each run starts again from the assembled blocks)
                auto run_pw = [&](int pw) -> rfm_status {
                    panel = pw;
                    return run_warps(nw);
                };
                std::vector<int> cands;
                for (int pw : {1, 2, 4, 8})
                    if (panel_fits(pw)) cands.push_back(pw);
                int best_pw = panel;
                rc = autotune_panel(F, pkind, st, run_pw, cands, &best_pw);
                panel = best_pw;
            }
        } else {
            rc = run_warps(nw);
        }
        if (rc != RFM_OK) return rc;
    }
    if (F.gather) {
        ProfScope ps("k_gather_kept", st);
        k_gather_kept<TM><<<nb, 256, 0, st>>>(F.blk, (const TM *)F.M, F.perm, F.rank, F.Op);
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    return RFM_OK;
}

// Cluster kernels visit the blocks largest first (the plan's order) unless
// RFM_OPT_QR_ORDER = 0; the factors do not depend on the order.
static int g_qr_order = 1;

const int32_t *qr_order_ptr(void *ws, const Layout &L) {
    return g_qr_order ? ws_ptr<int32_t>(ws, L.off_qord) : nullptr;
}

static FilterBufs system_bufs(const HostPlan &P, void *ws) {
    const Layout &L = P.L;
    FilterBufs F = {};
    F.blk = ws_ptr<BlkRec>(ws, L.off_blk);
    F.order = qr_order_ptr(ws, L);
    F.M = ws_ptr<char>(ws, L.off_M);
    F.W = ws_ptr<double>(ws, L.off_W);
    F.tau = ws_ptr<double>(ws, L.off_tau);
    F.perm = ws_ptr<int32_t>(ws, L.off_perm);
    F.rank = ws_ptr<int32_t>(ws, L.off_rank);
    F.r11 = ws_ptr<double>(ws, L.off_r11);
    F.Op = ws_ptr<double>(ws, L.off_op);
    F.Q32 = L.op == RFM_OP_Q32 ? ws_ptr<float>(ws, L.off_q32) : nullptr;
    F.Q64 = L.op == RFM_OP_Q64 ? F.Op : nullptr;
    F.gather = L.op == RFM_OP_AR64;
    F.n_blocks = L.n_blocks;
    F.max_m = L.max_m;
    F.max_K = L.max_K;
    F.fit = false;
    return F;
}

// Test hook: force the global-memory kernels (cluster sizes disabled).
static int g_force_global = 0;

rfm_status launch_filter_bufs(const FilterBufs &F0, bool fp32, double tol, cudaStream_t st) {
    if (F0.n_blocks == 0) return RFM_OK;
    FilterBufs F = F0;
    if (g_force_global) F.no_cluster = true;
    return fp32 ? launch_filter_t<float>(F, tol, st) : launch_filter_t<double>(F, tol, st);
}

rfm_status launch_filter(const HostPlan &P, void *ws, double tol, cudaStream_t st) {
    return launch_filter_bufs(system_bufs(P, ws), P.L.asm_prec == RFM_ASM_FP32, tol, st);
}

void set_force_global_filter(int on) { g_force_global = on; }
void set_autotune(int on) { g_autotune = on; }
void set_qr_double_float(int on) { g_qr_df = on; }
void set_qr_order(int on) { g_qr_order = on; }

}  // namespace rfm
