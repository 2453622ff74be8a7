// fit.cu -- learned warm start: from predicted solution values at every
// block's rows to a starting point y0 of the preconditioned LSQR.
//
// Per block j with kept features k_1..k_r (pivot order of the system's
// filter), window w_j and predictions u_hat_j at the block's rows:
//   V_j[i, c] = w_j(x_i) phi_{j k_c}(x_i)   (window-weighted feature values)
//   V_j P_j = Q_j R_Vj                      (QR with column pivoting,
//                                            truncated at tol_fit |R_11|)
// Local fit (fit_iters = 0): c_j = argmin ||V_j c - w_j u_hat_j||.
// Global fit (fit_iters > 0): the blended prediction u_bar(x_r) =
//   sum_j w_j(x_r) u_hat_j(x_r) at every collocation row is fitted by
//   sum_j V_j c_j through all blocks at once -- LSQR on the right-
//   preconditioned fitting system [Q_1 ... Q_J] z = u_bar (the explicit
//   operator of Proposition 3.1 for the value blocks), c_j = P_j R_Vj^-1 z_j.
// Either way y0_j = R_j c_j with R_j the system's filter factor, so that
// a = S^-1 y0 starts at the fitted coefficients.  V_j and its factors depend
// only on the decomposition and the features: rfm_fit_prepare forms them
// once.
#include "device.cuh"
#include "prof.cuh"

namespace rfm {

struct FitLayout {
    size_t off_phi, off_w, off_q, off_tau, off_perm, off_rank, off_r11, off_wrow, off_hbar, off_z, total;
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
    F.off_wrow = take((size_t)P.L.block_rows * 8);
    F.off_hbar = take((size_t)P.L.n_rows * 8);
    F.off_z = take((size_t)ncol * 8);
    F.total = o;
    return F;
}

size_t fit_workspace_bytes(const HostPlan &P) { return fit_layout(P).total; }

// V of every block over its kept columns (pivot order): window times feature
// value; zero columns from the block's rank on and zero padding rows; the
// window of every block row into wrow.  One CTA per 32-row tile.
__global__ void __launch_bounds__(256) k_fit_values(const InstRec *__restrict__ insts, const BlkRec *__restrict__ blks,
                                                    const int32_t *__restrict__ tile_blk,
                                                    const int32_t *__restrict__ tile_row,
                                                    const double *__restrict__ params, const int32_t *__restrict__ perm,
                                                    const int32_t *__restrict__ rank, double *__restrict__ Phi,
                                                    double *__restrict__ wrow) {
    __shared__ double s_s[32][3];
    __shared__ double s_w[32];
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
        double x[3] = {0, 0, 0}, w = 0.0;
        const int lr = r0 + lane;
        if (lr < B.m) {
            int kind, gcov[3];
            block_row_point(I, B, lr, x, &kind, gcov);
            double dw[3], d2w[3];
            window_nd(I, B.jd, x, &w, dw, d2w);
        }
        for (int i = 0; i < 3; ++i) s_s[lane][i] = i < I.dim ? (x[i] - B.mu[i]) / B.sig[i] : 0.0;
        s_w[lane] = w;
        if (lr < B.ldm) wrow[B.roff + lr] = w;
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
            v = s_w[lane] * tanh(z);
        }
        out[(int64_t)c * B.ldm] = v;
    }
}

// c = P_V R_V^-1 z (z: k entries in shared memory, FP64 back substitution),
// scattered into the system's pivot order, then y0 = R c.
__device__ void fit_finish_block(const BlkRec &B, int r, int k, const double *Wf, const int32_t *permf,
                                 const double *W, double *z, double *c, double *y0) {
    const int tid = threadIdx.x, ld = B.ldm, K = B.K;
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
    const double *R = W + B.moff;
    for (int i = tid; i < K; i += 256) {
        double s = 0.0;
        if (i < r)
            for (int j = i; j < r; ++j) s = fma(R[(int64_t)j * ld + i], c[j], s);
        y0[B.coff + i] = s;
    }
}

// Local fit, one CTA per block: z = Q_V^T (w u_hat), then fit_finish_block.
__global__ void __launch_bounds__(256) k_fit_local(const BlkRec *__restrict__ blks, const double *__restrict__ Qf,
                                                   const double *__restrict__ Wf, const int32_t *__restrict__ permf,
                                                   const int32_t *__restrict__ rankf, const double *__restrict__ W,
                                                   const int32_t *__restrict__ rank, const double *__restrict__ wrow,
                                                   const float *__restrict__ uhat, const float *__restrict__ iscale,
                                                   double *__restrict__ y0) {
    extern __shared__ double fs[];
    const BlkRec &B = blks[blockIdx.x];
    const int m = B.m, ld = B.ldm, K = B.K;
    const int r = rank[blockIdx.x], k = rankf[blockIdx.x];
    double *u = fs;          // ld
    double *z = u + ld;      // K
    double *c = z + K;       // K
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double sc = iscale ? (double)iscale[B.inst] : 1.0;
    for (int i = tid; i < m; i += 256) u[i] = wrow[B.roff + i] * ((double)uhat[B.roff + i] * sc);
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
    fit_finish_block(B, r, k, Wf, permf, W, z, c, y0);
}

// Global fit, after LSQR on the fitting system: z per block from zg.
__global__ void __launch_bounds__(256) k_fit_finish(const BlkRec *__restrict__ blks, const double *__restrict__ Wf,
                                                    const int32_t *__restrict__ permf, const int32_t *__restrict__ rankf,
                                                    const double *__restrict__ W, const int32_t *__restrict__ rank,
                                                    const double *__restrict__ zg, double *__restrict__ y0) {
    extern __shared__ double fs[];
    const BlkRec &B = blks[blockIdx.x];
    const int K = B.K, r = rank[blockIdx.x], k = rankf[blockIdx.x];
    double *z = fs;       // K
    double *c = z + K;    // K
    for (int t = threadIdx.x; t < K; t += 256) {
        z[t] = t < k ? zg[B.coff + t] : 0.0;
        c[t] = 0.0;
    }
    __syncthreads();
    fit_finish_block(B, r, k, Wf, permf, W, z, c, y0);
}

// u_bar at every collocation row: sum over the block rows holding it of
// w_j(x) u_hat_j(x) (same order as the rows' lists).
__global__ void k_fit_blend(const InstRec *__restrict__ insts, int n_inst, const int32_t *__restrict__ rowlist,
                            const double *__restrict__ wrow, const float *__restrict__ uhat,
                            const float *__restrict__ iscale, double *__restrict__ hbar, int64_t n_rows) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_rows; g += (int64_t)gridDim.x * blockDim.x) {
        int s = 0;
        while (s + 1 < n_inst && insts[s + 1].row0 <= g) ++s;
        const InstRec &I = insts[s];
        const int64_t r = g - I.row0;
        const int32_t *lst = rowlist + I.rl_off + r * I.C;
        double acc = 0.0;
        for (int e = 0; e < I.C; ++e) {
            const int q = lst[e];
            if (q >= 0) acc = fma(wrow[q], (double)uhat[q], acc);
        }
        hbar[g] = iscale ? acc * (double)iscale[s] : acc;
    }
}

rfm_status launch_fit_prepare(const HostPlan &P, void *ws, const double *params, double tol_fit, void *fws,
                              cudaStream_t st) {
    const Layout &L = P.L;
    if (L.op == RFM_OP_PLAIN) {
        set_error("rfm_fit_prepare: the system has no filter factors (plain operator)");
        return RFM_EINVAL;
    }
    for (int s = 0; s < L.n_inst; ++s)
        if (P.inst[s].depth != 1 || P.inst[s].act != RFM_ACT_TANH || P.inst[s].hard_bc != 0.0) {
            set_error("rfm_fit_prepare: the fit takes one-layer tanh networks without hard constraint");
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
            ws_ptr<int32_t>(ws, L.off_rank), Phi, ws_ptr<double>(fws, F.off_wrow));
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    FilterBufs B = {};
    B.blk = ws_ptr<BlkRec>(ws, L.off_blk);
    B.order = qr_order_ptr(ws, L);
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

rfm_status launch_lsqr_on(const HostPlan &P, void *ws, const double *Op, const int32_t *rank, const double *rhs,
                          int iters, double *z_out, rfm_lsqr_report *rep, cudaStream_t st);

rfm_status launch_warm_start(const HostPlan &P, void *ws, void *fws, const float *uhat, const float *iscale,
                             int fit_iters, double *y0, cudaStream_t st) {
    const Layout &L = P.L;
    if (L.n_blocks == 0) return RFM_OK;
    const FitLayout F = fit_layout(P);
    const int64_t ldmax = (L.max_m + kLdAlign - 1) / kLdAlign * kLdAlign;
    const BlkRec *dB = ws_ptr<BlkRec>(ws, L.off_blk);
    const double *Wf = ws_ptr<double>(fws, F.off_w);
    const int32_t *permf = ws_ptr<int32_t>(fws, F.off_perm), *rankf = ws_ptr<int32_t>(fws, F.off_rank);
    const double *W = ws_ptr<double>(ws, L.off_W);
    const int32_t *rank = ws_ptr<int32_t>(ws, L.off_rank);
    if (fit_iters <= 0) {
        const size_t smem = (size_t)(ldmax + 2 * L.max_K) * 8;
        if (smem > 200 * 1024) {
            set_error("rfm_warm_start: blocks of %lld rows and %lld features exceed the local fit's shared memory",
                      (long long)L.max_m, (long long)L.max_K);
            return RFM_EINVAL;
        }
        ProfScope ps("k_fit_local", st);
        RFM_CUDA_CHECK(cudaFuncSetAttribute(k_fit_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_fit_local<<<(unsigned)L.n_blocks, 256, smem, st>>>(dB, ws_ptr<double>(fws, F.off_q), Wf, permf, rankf, W,
                                                             rank, ws_ptr<double>(fws, F.off_wrow), uhat, iscale, y0);
        RFM_CUDA_CHECK(cudaGetLastError());
        return RFM_OK;
    }
    double *hbar = ws_ptr<double>(fws, F.off_hbar);
    double *zg = ws_ptr<double>(fws, F.off_z);
    {
        ProfScope ps("k_fit_blend", st);
        const int64_t n = L.n_rows;
        const unsigned g = (unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
        k_fit_blend<<<g < 1 ? 1 : g, 256, 0, st>>>(ws_ptr<InstRec>(ws, L.off_inst), L.n_inst,
                                                    ws_ptr<int32_t>(ws, L.off_rowlist),
                                                    ws_ptr<double>(fws, F.off_wrow), uhat, iscale, hbar, n);
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    rfm_status rc = launch_lsqr_on(P, ws, ws_ptr<double>(fws, F.off_q), rankf, hbar, fit_iters, zg, nullptr, st);
    if (rc != RFM_OK) return rc;
    ProfScope ps("k_fit_finish", st);
    const size_t smem = (size_t)2 * L.max_K * 8;
    k_fit_finish<<<(unsigned)L.n_blocks, 256, smem, st>>>(dB, Wf, permf, rankf, W, rank, zg, y0);
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
