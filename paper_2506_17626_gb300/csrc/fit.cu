// fit.cu -- learned warm start: from predicted solution values at every
// block's rows to a starting point y0 of the preconditioned LSQR.
//
// Per block j with kept features k_1..k_r (pivot order of the system's
// filter) and predictions u_hat at the block's rows:
//   Phi_j[i, c] = phi_{j k_c}(x_i)        (feature values, no window)
//   c_j = argmin ||Phi_j c - u_hat||      (QR with column pivoting of Phi_j,
//                                          truncated at tol_fit |R_11|)
//   y0_j = R_j c_j                         (R_j: the system's filter factor)
// so that a = S^-1 y0 starts at the fitted coefficients.  By the partition of
// unity, sum_j w_j phi_j c_j reproduces the predictions where every block
// fits them.  Phi_j and its factors depend only on the decomposition and the
// features: rfm_fit_prepare forms them once; rfm_warm_start then costs one
// transposed product with Q_hat(Phi_j) and two triangular passes per block.
#include "device.cuh"
#include "prof.cuh"

namespace rfm {

struct FitLayout {
    size_t off_phi, off_w, off_q, off_tau, off_perm, off_rank, off_r11, total;
    int64_t melem;
};

static FitLayout fit_layout(const HostPlan &P) {
    FitLayout F;
    int64_t melem = 0;
    for (int64_t b = 0; b < P.L.n_blocks; ++b) melem += (int64_t)P.blk[b].ldm * P.blk[b].K;
    F.melem = melem;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o += (bytes + 255) / 256 * 256;
        return at;
    };
    const int64_t ncol = P.L.n_cols, nb = P.L.n_blocks;
    F.off_phi = take((size_t)melem * 8);
    F.off_w = take((size_t)melem * 8);
    F.off_q = take((size_t)melem * 8);
    F.off_tau = take((size_t)ncol * 8);
    F.off_perm = take((size_t)ncol * 4);
    F.off_rank = take((size_t)nb * 4);
    F.off_r11 = take((size_t)nb * 8);
    F.total = o;
    return F;
}

size_t fit_workspace_bytes(const HostPlan &P) { return fit_layout(P).total; }

// Phi of every block over its kept columns (pivot order), zero columns from
// the block's rank on and zero padding rows; one CTA per 32-row tile.
__global__ void __launch_bounds__(256) k_fit_values(const InstRec *__restrict__ insts, const BlkRec *__restrict__ blks,
                                                    const int32_t *__restrict__ tile_blk,
                                                    const int32_t *__restrict__ tile_row,
                                                    const double *__restrict__ params, const int32_t *__restrict__ perm,
                                                    const int32_t *__restrict__ rank, double *__restrict__ Phi) {
    __shared__ double s_s[32][3];
    __shared__ BlkRec sB;
    __shared__ InstRec sI;
    const int tile = blockIdx.x;
    const int b = tile_blk[tile];
    if (threadIdx.x == 0) {
        sB = blks[b];
        sI = insts[sB.inst];
    }
    __syncthreads();
    const BlkRec &B = sB;
    const InstRec &I = sI;
    const int r0 = tile_row[tile];
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    if (wy == 0) {
        double x[3] = {0, 0, 0};
        const int lr = r0 + lane;
        if (lr < B.m) {
            int kind, gcov[3];
            block_row_point(I, B, lr, x, &kind, gcov);
        }
        for (int i = 0; i < 3; ++i) s_s[lane][i] = i < I.dim ? (x[i] - B.mu[i]) / B.sig[i] : 0.0;
    }
    __syncthreads();
    const int lr = r0 + lane;
    if (lr >= B.ldm) return;
    const int r = rank[b], d = I.dim;
    const double *prm = params + I.prm_off + (int64_t)B.j * B.K * (d + 1);
    double *out = Phi + B.moff + lr;
    for (int c = wy; c < B.K; c += 8) {
        double v = 0.0;
        if (lr < B.m && c < r) {
            const double *pk = prm + (int64_t)perm[B.coff + c] * (d + 1);
            double z = pk[d];
            for (int i = 0; i < d; ++i) z = fma(pk[i], s_s[lane][i], z);
            v = tanh(z);
        }
        out[(int64_t)c * B.ldm] = v;
    }
}

// One CTA per block: z = Q_hat(Phi)^T u_hat, R(Phi) c' = z, scatter c' by the
// fit's pivots into c, y0 = R c over the system's kept columns.
__global__ void __launch_bounds__(256) k_fit_apply(const BlkRec *__restrict__ blks, const double *__restrict__ Qf,
                                                   const double *__restrict__ Wf, const int32_t *__restrict__ permf,
                                                   const int32_t *__restrict__ rankf, const double *__restrict__ W,
                                                   const int32_t *__restrict__ rank, const float *__restrict__ uhat,
                                                   double *__restrict__ y0) {
    extern __shared__ double fs[];
    const BlkRec &B = blks[blockIdx.x];
    const int m = B.m, ld = B.ldm, K = B.K;
    const int r = rank[blockIdx.x], k = rankf[blockIdx.x];
    double *u = fs;          // m
    double *z = u + ld;      // K
    double *c = z + K;       // K
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < m; i += 256) u[i] = (double)uhat[B.roff + i];
    for (int t = tid; t < K; t += 256) c[t] = 0.0;
    __syncthreads();
    const double *Qb = Qf + B.moff;
    for (int t = warp; t < k; t += 8) {
        const double *q = Qb + (int64_t)t * ld;
        double s = 0.0;
        for (int i = lane; i < m; i += 32) s = fma(q[i], u[i], s);
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) z[t] = s;
    }
    __syncthreads();
    // back substitution with R(Phi) (upper triangle of the fit's QR work)
    const double *Rf = Wf + B.moff;
    for (int j = k - 1; j >= 0; --j) {
        if (tid == 0) z[j] = z[j] / Rf[(int64_t)j * ld + j];
        __syncthreads();
        const double xj = z[j];
        for (int i = tid; i < j; i += 256) z[i] = fma(-Rf[(int64_t)j * ld + i], xj, z[i]);
        __syncthreads();
    }
    for (int t = tid; t < k; t += 256) c[permf[B.coff + t]] = z[t];
    __syncthreads();
    // y0 = R c with R the system's filter factor (r x r, upper)
    const double *R = W + B.moff;
    for (int i = tid; i < K; i += 256) {
        double s = 0.0;
        if (i < r)
            for (int j = i; j < r; ++j) s = fma(R[(int64_t)j * ld + i], c[j], s);
        y0[B.coff + i] = s;
    }
}

rfm_status launch_fit_prepare(const HostPlan &P, void *ws, const double *params, double tol_fit, void *fws,
                              cudaStream_t st) {
    const Layout &L = P.L;
    if (L.op == RFM_OP_PLAIN) {
        set_error("rfm_fit_prepare: the system has no filter factors (plain operator)");
        return RFM_EINVAL;
    }
    if (L.n_blocks == 0) return RFM_OK;
    const FitLayout F = fit_layout(P);
    double *Phi = ws_ptr<double>(fws, F.off_phi);
    {
        ProfScope ps("k_fit_values", st);
        k_fit_values<<<(unsigned)L.n_tiles, 256, 0, st>>>(
            ws_ptr<InstRec>(ws, L.off_inst), ws_ptr<BlkRec>(ws, L.off_blk), ws_ptr<int32_t>(ws, L.off_tile),
            ws_ptr<int32_t>(ws, L.off_tile) + L.n_tiles, params, ws_ptr<int32_t>(ws, L.off_perm),
            ws_ptr<int32_t>(ws, L.off_rank), Phi);
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    FilterBufs B;
    B.blk = ws_ptr<BlkRec>(ws, L.off_blk);
    B.M = Phi;
    B.W = ws_ptr<double>(fws, F.off_w);
    B.tau = ws_ptr<double>(fws, F.off_tau);
    B.perm = ws_ptr<int32_t>(fws, F.off_perm);
    B.rank = ws_ptr<int32_t>(fws, F.off_rank);
    B.r11 = ws_ptr<double>(fws, F.off_r11);
    B.Op = ws_ptr<double>(fws, F.off_q);
    B.Q64 = B.Op;
    B.Q32 = nullptr;
    B.gather = false;
    B.fit = true;
    B.n_blocks = L.n_blocks;
    B.max_m = L.max_m;
    B.max_K = L.max_K;
    return launch_filter_bufs(B, false, tol_fit, st);
}

rfm_status launch_warm_start(const HostPlan &P, void *ws, void *fws, const float *uhat, double *y0, cudaStream_t st) {
    const Layout &L = P.L;
    if (L.n_blocks == 0) return RFM_OK;
    const FitLayout F = fit_layout(P);
    const int64_t ldmax = (L.max_m + kLdAlign - 1) / kLdAlign * kLdAlign;
    const size_t smem = (size_t)(ldmax + 2 * L.max_K) * 8;
    if (smem > 200 * 1024) {
        set_error("rfm_warm_start: blocks of %lld rows and %lld features exceed the kernel's shared memory",
                  (long long)L.max_m, (long long)L.max_K);
        return RFM_EINVAL;
    }
    ProfScope ps("k_fit_apply", st);
    RFM_CUDA_CHECK(cudaFuncSetAttribute(k_fit_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_fit_apply<<<(unsigned)L.n_blocks, 256, smem, st>>>(
        ws_ptr<BlkRec>(ws, L.off_blk), ws_ptr<double>(fws, F.off_q), ws_ptr<double>(fws, F.off_w),
        ws_ptr<int32_t>(fws, F.off_perm), ws_ptr<int32_t>(fws, F.off_rank), ws_ptr<double>(ws, L.off_W),
        ws_ptr<int32_t>(ws, L.off_rank), uhat, y0);
    RFM_CUDA_CHECK(cudaGetLastError());
    return RFM_OK;
}

// Network inputs at every block row: [ctx of the instance (n_ctx), centre of
// the block (dim), (x - centre) / half-width (dim)]; optionally the row's
// point (3 doubles).  Padding rows get zeros.
__global__ void __launch_bounds__(256) k_block_inputs(const InstRec *__restrict__ insts,
                                                      const BlkRec *__restrict__ blks,
                                                      const int32_t *__restrict__ tile_blk,
                                                      const int32_t *__restrict__ tile_row,
                                                      const float *__restrict__ ctx, int n_ctx,
                                                      float *__restrict__ X, double *__restrict__ pts) {
    const int tile = blockIdx.x;
    const BlkRec &B = blks[tile_blk[tile]];
    const InstRec &I = insts[B.inst];
    const int lr = tile_row[tile] + (threadIdx.x & 31);
    const int part = threadIdx.x >> 5;   // warp 0: point and inputs; others idle
    if (part != 0 || lr >= B.ldm) return;
    const int d = I.dim, nin = n_ctx + 2 * d;
    const int64_t row = B.roff + lr;
    double x[3] = {0, 0, 0};
    const bool live = lr < B.m;
    if (live) {
        int kind, gcov[3];
        block_row_point(I, B, lr, x, &kind, gcov);
    }
    float *xr = X + row * nin;
    for (int q = 0; q < n_ctx; ++q) xr[q] = live ? ctx[(int64_t)B.inst * n_ctx + q] : 0.f;
    for (int i = 0; i < d; ++i) {
        xr[n_ctx + i] = live ? (float)B.mu[i] : 0.f;
        xr[n_ctx + d + i] = live ? (float)((x[i] - B.mu[i]) / B.sig[i]) : 0.f;
    }
    if (pts)
        for (int i = 0; i < 3; ++i) pts[row * 3 + i] = live ? x[i] : 0.0;
}

rfm_status launch_block_inputs(const HostPlan &P, void *ws, const float *ctx, int n_ctx, float *X, double *pts,
                               cudaStream_t st) {
    const Layout &L = P.L;
    if (L.n_tiles == 0) return RFM_OK;
    ProfScope ps("k_block_inputs", st);
    k_block_inputs<<<(unsigned)L.n_tiles, 256, 0, st>>>(ws_ptr<InstRec>(ws, L.off_inst), ws_ptr<BlkRec>(ws, L.off_blk),
                                                        ws_ptr<int32_t>(ws, L.off_tile),
                                                        ws_ptr<int32_t>(ws, L.off_tile) + L.n_tiles, ctx, n_ctx, X,
                                                        pts);
    RFM_CUDA_CHECK(cudaGetLastError());
    return RFM_OK;
}

}  // namespace rfm
