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
#include <cooperative_groups.h>

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

}  // namespace rfm

namespace rfm {
// ---------------------------------------------------------------------------
// Cluster variant: the block lives in the shared memory of a cluster of C
// CTAs (thread-block cluster, distributed shared memory), distributed by
// columns: column position c belongs to CTA c mod C, slot c / C.  Per step:
//   argmax of the trailing norms (each CTA over its columns, then every CTA
//   reads the C candidates through DSMEM and takes the same winner), column
//   swap between the two owners through DSMEM, reflector formed by the owner
//   of column k, every CTA copies v from the owner's shared memory and updates
//   its own trailing columns.  Three cluster barriers per step; no global
//   memory traffic inside the factorisation.  Q_hat (when wanted) is then
//   accumulated backwards in the same shared memory, each CTA on its own
//   columns, reading the reflectors back from global memory.
// ---------------------------------------------------------------------------
namespace cg = cooperative_groups;

struct Cand {
    double v;
    int p, c;
};

template <typename TM, int C>
__global__ void __launch_bounds__(256) k_qrcp_cluster(const BlkRec *__restrict__ blks, const TM *__restrict__ M,
                                                      double *__restrict__ W, double *__restrict__ tau,
                                                      int32_t *__restrict__ perm_out, int32_t *__restrict__ rank_out,
                                                      double *__restrict__ r11_out, double tol, int nloc_max,
                                                      int ld_loc, double *__restrict__ Qout, float *__restrict__ Q32) {
    cg::cluster_group cl = cg::this_cluster();
    const int cr = (int)cl.block_rank();
    const int b = blockIdx.x / C;
    const BlkRec B = blks[b];
    const int m = B.m, K = B.K, ld = B.ldm;
    extern __shared__ __align__(16) double sm[];
    double *A = sm;                                  // nloc_max x ld_loc
    double *vbuf = A + (size_t)nloc_max * ld_loc;     // ld_loc
    double *cn = vbuf + ld_loc;                      // nloc_max
    double *cn0 = cn + nloc_max;                     // nloc_max
    int *perm = (int *)(cn0 + nloc_max);             // nloc_max
    __shared__ Cand cand;
    __shared__ Cand red[8];
    __shared__ double s_nx, s_tau, s_meta[2];
    __shared__ int s_pmeta;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nloc = (K - cr + C - 1) / C;   // columns owned by this CTA
    double *Wb = W + B.moff;

    // load owned columns (FP64) and their exact norms
    for (int l = warp; l < nloc; l += 8) {
        const int c = cr + C * l;
        const TM *src = M + B.moff + (int64_t)c * ld;
        double s = 0.0;
        for (int i = lane; i < m; i += 32) {
            double a = (double)src[i];
            A[(size_t)l * ld_loc + i] = a;
            s = fma(a, a, s);
        }
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            cn[l] = sqrt(s);
            cn0[l] = cn[l];
            perm[l] = c;
        }
    }
    __syncthreads();
    const int steps = m < K ? m : K;
    const double tol3z = sqrt(2.220446049250313e-16);
    double R11 = 0.0;
    int rank = steps;
    for (int k = 0; k < steps; ++k) {
        // 1. local candidate among owned positions c >= k
        double bv = -1.0;
        int bp = 0x7fffffff, bc = k;
        const int l0 = (k - cr + C - 1) / C > 0 ? (k - cr + C - 1) / C : 0;  // first slot with position >= k
        for (int l = l0 + tid; l < nloc; l += 256) {
            const int c = cr + C * l;
            if (better(cn[l], perm[l], bv, bp)) { bv = cn[l]; bp = perm[l]; bc = c; }
        }
        for (int o = 16; o; o >>= 1) {
            double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
            int p2 = __shfl_xor_sync(0xffffffffu, bp, o);
            int c2 = __shfl_xor_sync(0xffffffffu, bc, o);
            if (better(v2, p2, bv, bp)) { bv = v2; bp = p2; bc = c2; }
        }
        if (lane == 0) red[warp] = Cand{bv, bp, bc};
        __syncthreads();
        if (tid == 0) {
            Cand t = red[0];
            for (int w = 1; w < 8; ++w)
                if (better(red[w].v, red[w].p, t.v, t.p)) t = red[w];
            cand = t;
        }
        cl.sync();
        // 2. winner over the cluster (same in every CTA)
        Cand win = *cl.map_shared_rank(&cand, 0);
        for (int r = 1; r < C; ++r) {
            Cand t = *cl.map_shared_rank(&cand, r);
            if (better(t.v, t.p, win.v, win.p)) win = t;
        }
        const int piv = win.c;
        const int ok = k % C, lk = k / C, op = piv % C, lp = piv / C;
        // 3. swap positions k and piv
        if (piv != k) {
            if (ok == op) {
                if (cr == ok) {
                    for (int i = tid; i < m; i += 256) {
                        double t = A[(size_t)lk * ld_loc + i];
                        A[(size_t)lk * ld_loc + i] = A[(size_t)lp * ld_loc + i];
                        A[(size_t)lp * ld_loc + i] = t;
                    }
                    if (tid == 0) {
                        double t = cn[lk]; cn[lk] = cn[lp]; cn[lp] = t;
                        t = cn0[lk]; cn0[lk] = cn0[lp]; cn0[lp] = t;
                        int q = perm[lk]; perm[lk] = perm[lp]; perm[lp] = q;
                    }
                }
                cl.sync();
            } else {
                // fetch the partner's column into vbuf, then write it after the barrier
                const int mine = cr == ok ? lk : lp, other_cta = cr == ok ? op : ok, other_slot = cr == ok ? lp : lk;
                const bool part = cr == ok || cr == op;
                if (part) {
                    const double *rA = cl.map_shared_rank(A, other_cta);
                    for (int i = tid; i < m; i += 256) vbuf[i] = rA[(size_t)other_slot * ld_loc + i];
                    if (tid == 0) {
                        s_meta[0] = cl.map_shared_rank(cn, other_cta)[other_slot];
                        s_meta[1] = cl.map_shared_rank(cn0, other_cta)[other_slot];
                        s_pmeta = cl.map_shared_rank(perm, other_cta)[other_slot];
                    }
                }
                cl.sync();
                if (part) {
                    for (int i = tid; i < m; i += 256) A[(size_t)mine * ld_loc + i] = vbuf[i];
                    if (tid == 0) {
                        cn[mine] = s_meta[0];
                        cn0[mine] = s_meta[1];
                        perm[mine] = s_pmeta;
                    }
                }
                __syncthreads();
            }
        }
        // 4. reflector by the owner of position k
        if (cr == ok) {
            double s = 0.0;
            const double *x = A + (size_t)lk * ld_loc;
            for (int i = k + tid; i < m; i += 256) s = fma(x[i], x[i], s);
            for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) red[warp].v = s;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int w = 0; w < 8; ++w) t += red[w].v;
                s_nx = sqrt(t);
            }
            __syncthreads();
        }
        cl.sync();
        const double nx = *cl.map_shared_rank(&s_nx, ok);
        if (k == 0) R11 = nx;
        if (nx == 0.0 || nx < tol * R11) { rank = k; break; }
        if (cr == ok) {
            double *x = A + (size_t)lk * ld_loc;
            const double alpha = x[k];
            const double beta = alpha >= 0.0 ? -nx : nx;
            const double scale = 1.0 / (alpha - beta);
            for (int i = k + 1 + tid; i < m; i += 256) x[i] *= scale;
            __syncthreads();
            if (tid == 0) {
                x[k] = beta;
                s_tau = (beta - alpha) / beta;
                tau[B.coff + k] = s_tau;
            }
        }
        cl.sync();
        // 5. every CTA copies v (rows k+1..m) and tau from the owner
        const double tk = *cl.map_shared_rank(&s_tau, ok);
        {
            const double *rx = cl.map_shared_rank(A, ok) + (size_t)lk * ld_loc;
            for (int i = k + 1 + tid; i < m; i += 256) vbuf[i] = rx[i];
        }
        __syncthreads();
        // 6. update owned trailing columns c > k, downdate their norms
        const int l1 = (k + 1 - cr + C - 1) / C > 0 ? (k + 1 - cr + C - 1) / C : 0;
        for (int l = l1 + warp; l < nloc; l += 8) {
            double *a = A + (size_t)l * ld_loc;
            double d = 0.0;
            for (int i = k + 1 + lane; i < m; i += 32) d = fma(vbuf[i], a[i], d);
            for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            const double akc = a[k];
            d = tk * (akc + d);
            for (int i = k + 1 + lane; i < m; i += 32) a[i] = fma(-d, vbuf[i], a[i]);
            const double rkc = akc - d;
            __syncwarp();
            if (lane == 0) a[k] = rkc;
            double cc = cn[l];
            int recompute = 0;
            if (cc != 0.0) {
                double t = fabs(rkc) / cc;
                t = (1.0 + t) * (1.0 - t);
                t = t < 0.0 ? 0.0 : t;
                double rr = cc / cn0[l];
                if (t * rr * rr <= tol3z) recompute = 1;
                else cc = cc * sqrt(t);
            }
            if (recompute) {
                double e = 0.0;
                for (int i = k + 1 + lane; i < m; i += 32) e = fma(a[i], a[i], e);
                for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
                cc = sqrt(e);
                if (lane == 0) cn0[l] = cc;
            }
            if (lane == 0) cn[l] = cc;
        }
        __syncthreads();
    }
    // write R and the reflectors of the owned columns, the permutation, rank
    for (int l = warp; l < nloc; l += 8) {
        const int c = cr + C * l;
        for (int i = lane; i < m; i += 32) Wb[(int64_t)c * ld + i] = A[(size_t)l * ld_loc + i];
    }
    for (int l = tid; l < nloc; l += 256) perm_out[B.coff + cr + C * l] = perm[l];
    if (cr == 0 && tid == 0) {
        rank_out[b] = rank;
        r11_out[b] = R11;
    }
    if (!Qout && !Q32) {
        cl.sync();
        return;
    }
    // Q_hat = H_0 ... H_{r-1} [I_r; 0], owned columns c < r, in shared memory
    cl.sync();  // every owner has written its reflectors to global memory
    __threadfence();
    const int r = rank;
    const int nq = (r - cr + C - 1) / C > 0 ? (r - cr + C - 1) / C : 0;
    for (int l = warp; l < nq; l += 8) {
        const int c = cr + C * l;
        for (int i = lane; i < m; i += 32) A[(size_t)l * ld_loc + i] = (i == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int k = r - 1; k >= 0; --k) {
        const double *v = Wb + (int64_t)k * ld;
        for (int i = k + 1 + tid; i < m; i += 256) vbuf[i] = v[i];
        __syncthreads();
        const double tk = tau[B.coff + k];
        const int lq = (k - cr + C - 1) / C > 0 ? (k - cr + C - 1) / C : 0;
        for (int l = lq + warp; l < nq; l += 8) {
            double *q = A + (size_t)l * ld_loc;
            double d = 0.0;
            for (int i = k + 1 + lane; i < m; i += 32) d = fma(vbuf[i], q[i], d);
            for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            const double qk = q[k];
            d = tk * (qk + d);
            for (int i = k + 1 + lane; i < m; i += 32) q[i] = fma(-d, vbuf[i], q[i]);
            __syncwarp();
            if (lane == 0) q[k] = qk - d;
        }
        __syncthreads();
    }
    for (int l = warp; l < nq; l += 8) {
        const int c = cr + C * l;
        for (int i = lane; i < m; i += 32) {
            const double qv = A[(size_t)l * ld_loc + i];
            if (Q32) Q32[B.moff + (int64_t)c * ld + i] = (float)qv;
            else Qout[B.moff + (int64_t)c * ld + i] = qv;
        }
    }
}

template <typename TM, int C>
static rfm_status launch_cluster(const HostPlan &P, void *ws, double tol, int nloc, int ldl, size_t smem, double *Qout,
                                 float *Q32, cudaStream_t st) {
    const Layout &L = P.L;
    auto kern = k_qrcp_cluster<TM, C>;
    RFM_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(L.n_blocks * C));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    RFM_CUDA_CHECK(cudaLaunchKernelEx(&cfg, kern, (const BlkRec *)ws_ptr<BlkRec>(ws, L.off_blk),
                                      (const TM *)ws_ptr<TM>(ws, L.off_M), ws_ptr<double>(ws, L.off_W),
                                      ws_ptr<double>(ws, L.off_tau), ws_ptr<int32_t>(ws, L.off_perm),
                                      ws_ptr<int32_t>(ws, L.off_rank), ws_ptr<double>(ws, L.off_r11), tol, nloc, ldl,
                                      Qout, Q32));
    return RFM_OK;
}

// Shared-memory bytes of the cluster kernel for cluster size C.
static size_t cluster_smem(int64_t max_m, int64_t max_K, int C, int *nloc, int *ldl) {
    *ldl = (int)((max_m + 1) / 2 * 2);
    *nloc = (int)((max_K + C - 1) / C);
    return ((size_t)(*nloc) * (*ldl) + (size_t)(*ldl)) * 8 + (size_t)(*nloc) * 20 + 64;
}

template <typename TM>
static rfm_status launch_filter_t(const HostPlan &P, void *ws, double tol, cudaStream_t st) {
    const Layout &L = P.L;
    const unsigned nb = (unsigned)L.n_blocks;
    BlkRec *dB = ws_ptr<BlkRec>(ws, L.off_blk);
    double *W = ws_ptr<double>(ws, L.off_W);
    double *tau = ws_ptr<double>(ws, L.off_tau);
    int32_t *perm = ws_ptr<int32_t>(ws, L.off_perm);
    int32_t *rank = ws_ptr<int32_t>(ws, L.off_rank);
    double *r11 = ws_ptr<double>(ws, L.off_r11);
    double *Op = ws_ptr<double>(ws, L.off_op);
    float *Q32 = L.op == RFM_OP_Q32 ? ws_ptr<float>(ws, L.off_q32) : nullptr;
    double *Q64 = L.op == RFM_OP_Q64 ? Op : nullptr;
    const size_t kSmemCap = 220 * 1024;
    int C = 0, nloc = 0, ldl = 0;
    size_t smem = 0;
    for (int c : {1, 2, 4, 8}) {
        smem = cluster_smem(L.max_m, L.max_K, c, &nloc, &ldl);
        if (smem <= kSmemCap) { C = c; break; }
    }
    if (C > 0) {
        ProfScope ps("k_qrcp_cluster", st);
        rfm_status rc;
        switch (C) {
            case 1: rc = launch_cluster<TM, 1>(P, ws, tol, nloc, ldl, smem, Q64, Q32, st); break;
            case 2: rc = launch_cluster<TM, 2>(P, ws, tol, nloc, ldl, smem, Q64, Q32, st); break;
            case 4: rc = launch_cluster<TM, 4>(P, ws, tol, nloc, ldl, smem, Q64, Q32, st); break;
            default: rc = launch_cluster<TM, 8>(P, ws, tol, nloc, ldl, smem, Q64, Q32, st); break;
        }
        if (rc != RFM_OK) return rc;
    } else {
        const size_t sm = (size_t)L.max_K * (2 * sizeof(double) + sizeof(int));
        {
            ProfScope ps("k_qrcp", st);
            RFM_CUDA_CHECK(cudaFuncSetAttribute(k_qrcp<TM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            k_qrcp<TM><<<nb, 256, sm, st>>>(dB, ws_ptr<TM>(ws, L.off_M), W, tau, perm, rank, r11, tol);
            RFM_CUDA_CHECK(cudaGetLastError());
        }
        if (L.op != RFM_OP_AR64) {
            ProfScope ps("k_form_q", st);
            k_form_q<<<nb, 256, 0, st>>>(dB, W, tau, rank, Op, Q32);
            RFM_CUDA_CHECK(cudaGetLastError());
        }
    }
    if (L.op == RFM_OP_AR64) {
        ProfScope ps("k_gather_kept", st);
        k_gather_kept<TM><<<nb, 256, 0, st>>>(dB, ws_ptr<TM>(ws, L.off_M), perm, rank, Op);
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    return RFM_OK;
}

// Test hook: force the global-memory kernels (cluster sizes disabled).
static int g_force_global = 0;

rfm_status launch_filter(const HostPlan &P, void *ws, double tol, cudaStream_t st) {
    if (P.L.n_blocks == 0) return RFM_OK;
    if (g_force_global) {
        HostPlan Q = P;
        Q.L.max_m = 1 << 30;   // no cluster size fits
        return P.L.asm_prec == RFM_ASM_FP32 ? launch_filter_t<float>(Q, ws, tol, st)
                                            : launch_filter_t<double>(Q, ws, tol, st);
    }
    return P.L.asm_prec == RFM_ASM_FP32 ? launch_filter_t<float>(P, ws, tol, st)
                                        : launch_filter_t<double>(P, ws, tol, st);
}

void set_force_global_filter(int on) { g_force_global = on; }

}  // namespace rfm
