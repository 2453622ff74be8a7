// api.cu -- the extern "C" entry points declared in include/rfm.h.
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "common.cuh"
#include "prof.cuh"

namespace rfm {
const char *last_error();
rfm_status launch_assemble(const HostPlan &P, void *ws, const double *params, cudaStream_t st);
rfm_status launch_filter(const HostPlan &P, void *ws, double tol, cudaStream_t st);
rfm_status launch_lsqr(const HostPlan &P, void *ws, const rfm_lsqr_opts *opts, const double *y0, double *y_out,
                       double *a_out, rfm_lsqr_report *rep, cudaStream_t st);
rfm_status launch_coefficients(const HostPlan &P, void *ws, const double *y, double *a_out, cudaStream_t st,
                               int nsets = 1);
rfm_status launch_residual(const HostPlan &P, void *ws, const double *a, double *r_out, double *rnorm,
                           cudaStream_t st);
size_t multi_workspace_bytes(const HostPlan &P, int R);
rfm_status launch_lsqr_multi(const HostPlan &P, void *ws, const rfm_lsqr_opts *opts, int R, const double *H,
                             const double *Y0, double *A, rfm_lsqr_report *rep, void *mws, cudaStream_t st);
rfm_status launch_rhs_many(const InstRec *recs, int R, int64_t N, double *H, void *scratch, cudaStream_t st);
void set_force_global_filter(int on);
void set_autotune(int on);
void set_qr_double_float(int on);
void set_lsqr_stall(int v);
void set_mlp_tensor_cores(int on);
void set_qr_order(int on);
void set_mlp_tc_threads(int threads);
void set_lsqr_lag(int tenths);
void set_multi_tc(int v);
void set_qr_warps(int v);
void set_qr_panel(int v);
rfm_status launch_eval_noalloc(const HostPlan &P, const double *params, const double *a, const double *X,
                               const int64_t *pt_off, double *u, double *err, cudaStream_t st);
rfm_status launch_eval(const HostPlan &P, void *ws, const double *params, const double *a, const double *X,
                       const int64_t *pt_off, double *u, double *err, cudaStream_t st);
size_t fit_workspace_bytes(const HostPlan &P);
rfm_status launch_fit_prepare(const HostPlan &P, void *ws, const double *params, double tol_fit, void *fws,
                              cudaStream_t st);
rfm_status launch_warm_start(const HostPlan &P, void *ws, void *fws, const float *uhat, const float *iscale,
                             int fit_iters, double *y0, cudaStream_t st);
rfm_status launch_block_inputs(const HostPlan &P, void *ws, const float *ctx, int n_ctx, float *X, double *pts,
                               cudaStream_t st);
rfm_status mlp_nparams(const rfm_mlp *net, int64_t *np);
rfm_status mlp_workspace(const rfm_mlp *net, size_t *bytes);
rfm_status launch_mlp_forward(const rfm_mlp *net, const float *theta, const float *X, int64_t n, float *Y,
                              cudaStream_t st);
rfm_status mlp_train_size(const rfm_mlp *net, int batch, size_t *bytes);
rfm_status launch_mlp_train(const rfm_mlp *net, float *theta, float *m, float *v, const float *X, const float *T,
                            const int64_t *order, int batch, int n_steps, int t0, const float *lr, float b1, float b2,
                            float eps, float *loss, void *ws, size_t ws_bytes, cudaStream_t st);
rfm_status launch_mlp_grad(const rfm_mlp *net, const float *theta, const float *X, const float *T, int64_t n,
                           float *grad, float *loss, void *ws, size_t ws_bytes, cudaStream_t st);
rfm_status launch_adam(int64_t n, float *theta, float *m, float *v, const float *g, int t, float lr, float b1,
                       float b2, float eps, cudaStream_t st);

namespace {
// RAII holder of a host plan for one call.
struct Plan {
    HostPlan p;
    bool ok = false;
    rfm_status rc = RFM_OK;
    Plan(const rfm_problem *probs, int n, const rfm_config *cfg) {
        char err[512] = {0};
        rc = build_plan(probs, n, cfg, &p, err, sizeof(err));
        ok = rc == RFM_OK;
        if (!ok) set_error("%s", err);
    }
    ~Plan() {
        if (ok) free_plan(&p);
    }
};

rfm_status check_ws(const Layout &L, const void *ws, size_t bytes) {
    if (!ws) {
        set_error("workspace pointer is NULL");
        return RFM_EINVAL;
    }
    if (((uintptr_t)ws & 255) != 0) {
        set_error("workspace must be 256-byte aligned");
        return RFM_EINVAL;
    }
    if (bytes < L.total) {
        set_error("workspace has %zu bytes, the system needs %zu", bytes, L.total);
        return RFM_ENOSPACE;
    }
    return RFM_OK;
}
}  // namespace
}  // namespace rfm

using namespace rfm;

#define RFM_GUARD_BEGIN try {
#define RFM_GUARD_END                                   \
    }                                                   \
    catch (const std::bad_alloc &) {                    \
        set_error("host allocation failed");            \
        return RFM_EINVAL;                              \
    }                                                   \
    catch (...) {                                       \
        set_error("unexpected host exception");         \
        return RFM_EINVAL;                              \
    }

extern "C" {

int rfm_abi_version(void) { return RFM_ABI_VERSION; }

const char *rfm_last_error(void) { return rfm::last_error(); }

rfm_status rfm_problem_size(const rfm_problem *probs, int n_inst, const rfm_config *cfg, rfm_sizes *out) {
    RFM_GUARD_BEGIN
    if (!out) {
        set_error("rfm_problem_size: out is NULL");
        return RFM_EINVAL;
    }
    Plan P(probs, n_inst, cfg);
    if (!P.ok) return P.rc;
    const Layout &L = P.p.L;
    out->n_inst = L.n_inst;
    out->n_blocks = L.n_blocks;
    out->n_rows = L.n_rows;
    out->n_cols = L.n_cols;
    out->block_rows = L.block_rows;
    out->max_block_rows = L.max_m;
    out->max_K = L.max_K;
    out->workspace_bytes = (int64_t)L.total;
    return RFM_OK;
    RFM_GUARD_END
}

rfm_status rfm_assemble(const rfm_problem *probs, int n_inst, const rfm_config *cfg, const double *d_params,
                        void *d_ws, size_t ws_bytes, void *stream) {
    RFM_GUARD_BEGIN
    Plan P(probs, n_inst, cfg);
    if (!P.ok) return P.rc;
    const Layout &L = P.p.L;
    rfm_status rc = check_ws(L, d_ws, ws_bytes);
    if (rc != RFM_OK) return rc;
    if (!d_params) {
        set_error("rfm_assemble: d_params is NULL");
        return RFM_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    RFM_CUDA_CHECK(cudaMemcpyAsync(ws_ptr<void>(d_ws, L.off_inst), P.p.inst, sizeof(InstRec) * L.n_inst,
                                   cudaMemcpyHostToDevice, st));
    if (L.n_blocks) {
        RFM_CUDA_CHECK(cudaMemcpyAsync(ws_ptr<void>(d_ws, L.off_blk), P.p.blk, sizeof(BlkRec) * L.n_blocks,
                                       cudaMemcpyHostToDevice, st));
        RFM_CUDA_CHECK(cudaMemcpyAsync(ws_ptr<void>(d_ws, L.off_qord), P.p.qr_order, sizeof(int32_t) * L.n_blocks,
                                       cudaMemcpyHostToDevice, st));
    }
    if (L.n_tiles) {
        RFM_CUDA_CHECK(cudaMemcpyAsync(ws_ptr<void>(d_ws, L.off_tile), P.p.tile_blk, sizeof(int32_t) * L.n_tiles,
                                       cudaMemcpyHostToDevice, st));
        RFM_CUDA_CHECK(cudaMemcpyAsync(ws_ptr<int32_t>(d_ws, L.off_tile) + L.n_tiles, P.p.tile_row,
                                       sizeof(int32_t) * L.n_tiles, cudaMemcpyHostToDevice, st));
    }
    if (L.n_cov)
        RFM_CUDA_CHECK(cudaMemcpyAsync(ws_ptr<void>(d_ws, L.off_cov), P.p.cov, sizeof(int32_t) * L.n_cov,
                                       cudaMemcpyHostToDevice, st));
    if (L.n_fwd_items)
        RFM_CUDA_CHECK(cudaMemcpyAsync(ws_ptr<void>(d_ws, L.off_fwd_items), P.p.fwd_items,
                                       sizeof(int32_t) * 2 * L.n_fwd_items, cudaMemcpyHostToDevice, st));
    if (L.n_col_items)
        RFM_CUDA_CHECK(cudaMemcpyAsync(ws_ptr<void>(d_ws, L.off_col_items), P.p.col_items,
                                       sizeof(int32_t) * 2 * L.n_col_items, cudaMemcpyHostToDevice, st));
    return launch_assemble(P.p, d_ws, d_params, st);
    RFM_GUARD_END
}

rfm_status rfm_rrqr_filter(const rfm_problem *probs, int n_inst, const rfm_config *cfg, void *d_ws, size_t ws_bytes,
                           int32_t *d_rank, int32_t *d_perm, void *stream) {
    RFM_GUARD_BEGIN
    Plan P(probs, n_inst, cfg);
    if (!P.ok) return P.rc;
    const Layout &L = P.p.L;
    rfm_status rc = check_ws(L, d_ws, ws_bytes);
    if (rc != RFM_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (L.op != RFM_OP_PLAIN) {
        rc = launch_filter(P.p, d_ws, cfg->tol, st);
        if (rc != RFM_OK) return rc;
    }
    if (d_rank && L.n_blocks) {
        if (L.op == RFM_OP_PLAIN) {
            set_error("rfm_rrqr_filter: no ranks with RFM_OP_PLAIN");
            return RFM_EINVAL;
        }
        RFM_CUDA_CHECK(cudaMemcpyAsync(d_rank, ws_ptr<void>(d_ws, L.off_rank), sizeof(int32_t) * L.n_blocks,
                                       cudaMemcpyDeviceToDevice, st));
    }
    if (d_perm && L.n_cols && L.op != RFM_OP_PLAIN)
        RFM_CUDA_CHECK(cudaMemcpyAsync(d_perm, ws_ptr<void>(d_ws, L.off_perm), sizeof(int32_t) * L.n_cols,
                                       cudaMemcpyDeviceToDevice, st));
    return RFM_OK;
    RFM_GUARD_END
}

rfm_status rfm_lsqr_solve(const rfm_problem *probs, int n_inst, const rfm_config *cfg, const rfm_lsqr_opts *opts,
                          const double *d_y0, double *d_y, double *d_a, rfm_lsqr_report *d_report, void *d_ws,
                          size_t ws_bytes, void *stream) {
    RFM_GUARD_BEGIN
    Plan P(probs, n_inst, cfg);
    if (!P.ok) return P.rc;
    const Layout &L = P.p.L;
    rfm_status rc = check_ws(L, d_ws, ws_bytes);
    if (rc != RFM_OK) return rc;
    if (!opts || !d_a || opts->max_iter < 0 || !(opts->atol >= 0.0) || !(opts->btol >= 0.0)) {
        set_error("rfm_lsqr_solve: need opts (max_iter >= 0, atol, btol >= 0) and d_a");
        return RFM_EINVAL;
    }
    return launch_lsqr(P.p, d_ws, opts, d_y0, d_y, d_a, d_report, (cudaStream_t)stream);
    RFM_GUARD_END
}

rfm_status rfm_coefficients(const rfm_problem *probs, int n_inst, const rfm_config *cfg, const double *d_y,
                            double *d_a, void *d_ws, size_t ws_bytes, void *stream) {
    RFM_GUARD_BEGIN
    Plan P(probs, n_inst, cfg);
    if (!P.ok) return P.rc;
    rfm_status rc = check_ws(P.p.L, d_ws, ws_bytes);
    if (rc != RFM_OK) return rc;
    if (!d_y || !d_a) {
        set_error("rfm_coefficients: null argument");
        return RFM_EINVAL;
    }
    return launch_coefficients(P.p, d_ws, d_y, d_a, (cudaStream_t)stream);
    RFM_GUARD_END
}

rfm_status rfm_residual(const rfm_problem *probs, int n_inst, const rfm_config *cfg, const double *d_a, double *d_r,
                        double *d_rnorm, void *d_ws, size_t ws_bytes, void *stream) {
    RFM_GUARD_BEGIN
    Plan P(probs, n_inst, cfg);
    if (!P.ok) return P.rc;
    rfm_status rc = check_ws(P.p.L, d_ws, ws_bytes);
    if (rc != RFM_OK) return rc;
    if (!d_a) {
        set_error("rfm_residual: d_a is NULL");
        return RFM_EINVAL;
    }
    return launch_residual(P.p, d_ws, d_a, d_r, d_rnorm, (cudaStream_t)stream);
    RFM_GUARD_END
}

rfm_status rfm_lsqr_multi_size(const rfm_problem *prob, const rfm_config *cfg, int nrhs, size_t *bytes) {
    RFM_GUARD_BEGIN
    Plan P(prob, 1, cfg);
    if (!P.ok) return P.rc;
    if (!bytes || nrhs < 1 || nrhs > 256) {
        set_error("rfm_lsqr_multi_size: need bytes and 1 <= nrhs <= 256");
        return RFM_EINVAL;
    }
    *bytes = multi_workspace_bytes(P.p, nrhs);
    return RFM_OK;
    RFM_GUARD_END
}

static rfm_status check_mws(const HostPlan &P, int nrhs, const void *mws, size_t bytes) {
    if (!mws || ((uintptr_t)mws & 255)) {
        set_error("multi-right-hand-side workspace must be a 256-byte aligned device pointer");
        return RFM_EINVAL;
    }
    if (bytes < multi_workspace_bytes(P, nrhs)) {
        set_error("multi-right-hand-side workspace has %zu bytes, %zu needed", bytes, multi_workspace_bytes(P, nrhs));
        return RFM_ENOSPACE;
    }
    return RFM_OK;
}

// Data sets of one family: everything but the data (family, n_modes, fam) equal.
static bool same_layout(const rfm_problem &a, const rfm_problem &b) {
    rfm_problem x = a, y = b;
    x.family = y.family = 0;
    x.n_modes = y.n_modes = 0;
    memset(x.fam, 0, sizeof(x.fam));
    memset(y.fam, 0, sizeof(y.fam));
    if (a.pde == RFM_PDE_OSC) {   // the oscillator's coefficients are part of the operator
        memcpy(x.fam, a.fam, 3 * sizeof(double));
        memcpy(y.fam, b.fam, 3 * sizeof(double));
    }
    return memcmp(&x, &y, sizeof(rfm_problem)) == 0;
}

rfm_status rfm_rhs_many(const rfm_problem *probs, int nrhs, const rfm_config *cfg, double *d_H, void *d_mws,
                        size_t mws_bytes, void *stream) {
    RFM_GUARD_BEGIN
    if (!probs || nrhs < 1 || nrhs > 256 || !d_H) {
        set_error("rfm_rhs_many: need probs, 1 <= nrhs <= 256 and d_H");
        return RFM_EINVAL;
    }
    Plan P0(probs, 1, cfg);
    if (!P0.ok) return P0.rc;
    rfm_status rc = check_mws(P0.p, nrhs, d_mws, mws_bytes);
    if (rc != RFM_OK) return rc;
    std::vector<InstRec> recs((size_t)nrhs);
    for (int j = 0; j < nrhs; ++j) {
        if (!same_layout(probs[0], probs[j])) {
            set_error("rfm_rhs_many: data set %d differs from set 0 in more than its data", j);
            return RFM_EINVAL;
        }
        Plan Pj(probs + j, 1, cfg);
        if (!Pj.ok) return Pj.rc;
        recs[(size_t)j] = Pj.p.inst[0];
    }
    return launch_rhs_many(recs.data(), nrhs, P0.p.L.n_rows, d_H, d_mws, (cudaStream_t)stream);
    RFM_GUARD_END
}

rfm_status rfm_lsqr_multi(const rfm_problem *prob, const rfm_config *cfg, const rfm_lsqr_opts *opts, int nrhs,
                          const double *d_H, const double *d_Y0, double *d_A, rfm_lsqr_report *d_report, void *d_ws,
                          size_t ws_bytes, void *d_mws, size_t mws_bytes, void *stream) {
    RFM_GUARD_BEGIN
    Plan P(prob, 1, cfg);
    if (!P.ok) return P.rc;
    rfm_status rc = check_ws(P.p.L, d_ws, ws_bytes);
    if (rc != RFM_OK) return rc;
    if (nrhs < 1 || nrhs > 256 || !d_H || !d_A || !opts || opts->max_iter < 0 || !(opts->atol >= 0.0) ||
        !(opts->btol >= 0.0)) {
        set_error("rfm_lsqr_multi: need 1 <= nrhs <= 256, d_H, d_A and opts (max_iter >= 0, atol, btol >= 0)");
        return RFM_EINVAL;
    }
    rc = check_mws(P.p, nrhs, d_mws, mws_bytes);
    if (rc != RFM_OK) return rc;
    return launch_lsqr_multi(P.p, d_ws, opts, nrhs, d_H, d_Y0, d_A, d_report, d_mws, (cudaStream_t)stream);
    RFM_GUARD_END
}

rfm_status rfm_set_option(int option, int value) {
    if (option == RFM_OPT_FILTER_KERNEL && (value == 0 || value == 1)) {
        set_force_global_filter(value);
        return RFM_OK;
    }
    if (option == RFM_OPT_AUTOTUNE && (value == 0 || value == 1)) {
        set_autotune(value);
        return RFM_OK;
    }
    if (option == RFM_OPT_QR_DOUBLE_FLOAT && value >= 0 && value <= 2) {
        set_qr_double_float(value);
        return RFM_OK;
    }
    if (option == RFM_OPT_LSQR_STALL && value >= 0 && value <= 2) {
        set_lsqr_stall(value);
        return RFM_OK;
    }
    if (option == RFM_OPT_MLP_TENSOR_CORES && (value == 0 || value == 1)) {
        set_mlp_tensor_cores(value);
        return RFM_OK;
    }
    if (option == RFM_OPT_QR_ORDER && (value == 0 || value == 1)) {
        set_qr_order(value);
        return RFM_OK;
    }
    if (option == RFM_OPT_LSQR_LAG && value >= 0 && value <= 100) {
        set_lsqr_lag(value);
        return RFM_OK;
    }
    if (option == RFM_OPT_QR_WARPS && (value == 4 || value == 8 || value == 16 || value == 32)) {
        set_qr_warps(value);
        return RFM_OK;
    }
    if (option == RFM_OPT_QR_PANEL && (value == 1 || value == 2 || value == 4 || value == 8)) {
        set_qr_panel(value);
        return RFM_OK;
    }
    if (option == RFM_OPT_MULTI_TENSOR_CORES && (value == 0 || value == 1)) {
        set_multi_tc(value);
        return RFM_OK;
    }
    if (option == RFM_OPT_MLP_TC_THREADS && (value == 256 || value == 512)) {
        set_mlp_tc_threads(value);
        return RFM_OK;
    }
    set_error("rfm_set_option: unknown option %d or value %d", option, value);
    return RFM_EINVAL;
}

rfm_status rfm_profile_enable(int on) {
    prof_enable(on != 0);
    return RFM_OK;
}

rfm_status rfm_profile_reset(void) {
    prof_reset();
    return RFM_OK;
}

int rfm_profile_read(const char **names, int64_t *launches, double *ms, int max) {
    try {
        return prof_read(names, launches, ms, max);
    } catch (...) {
        return -1;
    }
}

rfm_status rfm_eval(const rfm_problem *probs, int n_inst, const rfm_config *cfg, const double *d_params,
                    const double *d_a, const double *d_x, const int64_t *h_pt_off, double *d_u, double *d_err,
                    void *d_ws, size_t ws_bytes, void *stream) {
    RFM_GUARD_BEGIN
    Plan P(probs, n_inst, cfg);
    if (!P.ok) return P.rc;
    const Layout &L = P.p.L;
    rfm_status rc = check_ws(L, d_ws, ws_bytes);
    if (rc != RFM_OK) return rc;
    if (!d_params || !d_a || !d_x || !h_pt_off || !d_u) {
        set_error("rfm_eval: null argument");
        return RFM_EINVAL;
    }
    return launch_eval(P.p, d_ws, d_params, d_a, d_x, h_pt_off, d_u, d_err, (cudaStream_t)stream);
    RFM_GUARD_END
}

rfm_status rfm_eval_noalloc(const rfm_problem *probs, int n_inst, const double *d_params, const double *d_a,
                            const double *d_x, const int64_t *h_pt_off, double *d_u, double *d_err, void *stream) {
    RFM_GUARD_BEGIN
    const rfm_config cfg = {RFM_ASM_FP64, RFM_OP_AR64, 0.0};
    Plan P(probs, n_inst, &cfg);
    if (!P.ok) return P.rc;
    if (!d_params || !d_a || !d_x || !h_pt_off || !d_u) {
        set_error("rfm_eval_noalloc: null argument");
        return RFM_EINVAL;
    }
    return launch_eval_noalloc(P.p, d_params, d_a, d_x, h_pt_off, d_u, d_err, (cudaStream_t)stream);
    RFM_GUARD_END
}

rfm_status rfm_block_info(const rfm_problem *probs, int n_inst, const rfm_config *cfg, int64_t block, int64_t *m,
                          int64_t *ld, int64_t *moff, int64_t *roff) {
    RFM_GUARD_BEGIN
    Plan P(probs, n_inst, cfg);
    if (!P.ok) return P.rc;
    if (block < 0 || block >= P.p.L.n_blocks) {
        set_error("rfm_block_info: block %lld out of range", (long long)block);
        return RFM_EINVAL;
    }
    const BlkRec &B = P.p.blk[block];
    if (m) *m = B.m;
    if (ld) *ld = B.ldm;
    if (moff) *moff = B.moff;
    if (roff) *roff = B.roff;
    return RFM_OK;
    RFM_GUARD_END
}

rfm_status rfm_block_table(const rfm_problem *probs, int n_inst, const rfm_config *cfg, int64_t *m, int64_t *ld,
                           int64_t *moff, int64_t *roff) {
    RFM_GUARD_BEGIN
    Plan P(probs, n_inst, cfg);
    if (!P.ok) return P.rc;
    for (int64_t b = 0; b < P.p.L.n_blocks; ++b) {
        const BlkRec &B = P.p.blk[b];
        if (m) m[b] = B.m;
        if (ld) ld[b] = B.ldm;
        if (moff) moff[b] = B.moff;
        if (roff) roff[b] = B.roff;
    }
    return RFM_OK;
    RFM_GUARD_END
}

rfm_status rfm_block_rows(const rfm_problem *probs, int n_inst, const rfm_config *cfg, int64_t block,
                          int64_t *rows) {
    RFM_GUARD_BEGIN
    Plan P(probs, n_inst, cfg);
    if (!P.ok) return P.rc;
    if (block < 0 || block >= P.p.L.n_blocks || !rows) {
        set_error("rfm_block_rows: block %lld out of range or rows NULL", (long long)block);
        return RFM_EINVAL;
    }
    host_block_rows(P.p, block, rows);
    return RFM_OK;
    RFM_GUARD_END
}

rfm_status rfm_qr_order(const rfm_problem *probs, int n_inst, const rfm_config *cfg, int32_t *order) {
    RFM_GUARD_BEGIN
    Plan P(probs, n_inst, cfg);
    if (!P.ok) return P.rc;
    if (!order) {
        set_error("rfm_qr_order: order is NULL");
        return RFM_EINVAL;
    }
    if (P.p.L.n_blocks) memcpy(order, P.p.qr_order, sizeof(int32_t) * P.p.L.n_blocks);
    return RFM_OK;
    RFM_GUARD_END
}

rfm_status rfm_workspace_view(const rfm_problem *probs, int n_inst, const rfm_config *cfg, void *d_ws, int which,
                              void **ptr) {
    RFM_GUARD_BEGIN
    Plan P(probs, n_inst, cfg);
    if (!P.ok) return P.rc;
    const Layout &L = P.p.L;
    size_t off;
    switch (which) {
        case 0: off = L.off_M; break;
        case 1: off = L.off_h; break;
        case 2: off = L.off_grow; break;
        case 3: off = L.off_W; break;
        case 4: off = L.off_r11; break;
        case 5: off = L.op == RFM_OP_Q32 ? L.off_q32 : L.off_op; break;
        default: set_error("rfm_workspace_view: unknown view %d", which); return RFM_EINVAL;
    }
    if (!ptr) {
        set_error("rfm_workspace_view: ptr is NULL");
        return RFM_EINVAL;
    }
    *ptr = ws_ptr<void>(d_ws, off);
    return RFM_OK;
    RFM_GUARD_END
}

rfm_status rfm_block_inputs(const rfm_problem *probs, int n_inst, const rfm_config *cfg, const float *d_ctx,
                            int n_ctx, float *d_x, double *d_pts, void *d_ws, size_t ws_bytes, void *stream) {
    RFM_GUARD_BEGIN
    Plan P(probs, n_inst, cfg);
    if (!P.ok) return P.rc;
    rfm_status rc = check_ws(P.p.L, d_ws, ws_bytes);
    if (rc != RFM_OK) return rc;
    if (n_ctx < 0 || n_ctx > 64 || (n_ctx > 0 && !d_ctx) || !d_x) {
        set_error("rfm_block_inputs: need 0 <= n_ctx <= 64, d_ctx when n_ctx > 0, and d_x");
        return RFM_EINVAL;
    }
    return launch_block_inputs(P.p, d_ws, d_ctx, n_ctx, d_x, d_pts, (cudaStream_t)stream);
    RFM_GUARD_END
}

rfm_status rfm_fit_size(const rfm_problem *probs, int n_inst, const rfm_config *cfg, size_t *bytes) {
    RFM_GUARD_BEGIN
    Plan P(probs, n_inst, cfg);
    if (!P.ok) return P.rc;
    if (!bytes) {
        set_error("rfm_fit_size: bytes is NULL");
        return RFM_EINVAL;
    }
    *bytes = fit_workspace_bytes(P.p);
    return RFM_OK;
    RFM_GUARD_END
}

static rfm_status check_fit_ws(const HostPlan &P, const void *fws, size_t fit_bytes) {
    if (!fws || ((uintptr_t)fws & 255)) {
        set_error("fit workspace must be a 256-byte aligned device pointer");
        return RFM_EINVAL;
    }
    if (fit_bytes < fit_workspace_bytes(P)) {
        set_error("fit workspace has %zu bytes, the system needs %zu", fit_bytes, fit_workspace_bytes(P));
        return RFM_ENOSPACE;
    }
    return RFM_OK;
}

rfm_status rfm_fit_prepare(const rfm_problem *probs, int n_inst, const rfm_config *cfg, const double *d_params,
                           double tol_fit, void *d_ws, size_t ws_bytes, void *d_fit_ws, size_t fit_bytes,
                           void *stream) {
    RFM_GUARD_BEGIN
    Plan P(probs, n_inst, cfg);
    if (!P.ok) return P.rc;
    rfm_status rc = check_ws(P.p.L, d_ws, ws_bytes);
    if (rc != RFM_OK) return rc;
    rc = check_fit_ws(P.p, d_fit_ws, fit_bytes);
    if (rc != RFM_OK) return rc;
    if (!d_params || !(tol_fit >= 0.0 && tol_fit < 1.0)) {
        set_error("rfm_fit_prepare: need d_params and 0 <= tol_fit < 1");
        return RFM_EINVAL;
    }
    return launch_fit_prepare(P.p, d_ws, d_params, tol_fit, d_fit_ws, (cudaStream_t)stream);
    RFM_GUARD_END
}

rfm_status rfm_warm_start(const rfm_problem *probs, int n_inst, const rfm_config *cfg, const float *d_uhat,
                          const float *d_inst_scale, int fit_iters, double *d_y0, void *d_ws, size_t ws_bytes,
                          void *d_fit_ws, size_t fit_bytes, void *stream) {
    RFM_GUARD_BEGIN
    Plan P(probs, n_inst, cfg);
    if (!P.ok) return P.rc;
    rfm_status rc = check_ws(P.p.L, d_ws, ws_bytes);
    if (rc != RFM_OK) return rc;
    rc = check_fit_ws(P.p, d_fit_ws, fit_bytes);
    if (rc != RFM_OK) return rc;
    if (!d_uhat || !d_y0) {
        set_error("rfm_warm_start: null argument");
        return RFM_EINVAL;
    }
    if (fit_iters < 0) {
        set_error("rfm_warm_start: fit_iters must be >= 0");
        return RFM_EINVAL;
    }
    return launch_warm_start(P.p, d_ws, d_fit_ws, d_uhat, d_inst_scale, fit_iters, d_y0, (cudaStream_t)stream);
    RFM_GUARD_END
}

rfm_status rfm_mlp_size(const rfm_mlp *net, int64_t *n_params, size_t *ws_bytes) {
    RFM_GUARD_BEGIN
    int64_t np = 0;
    size_t wb = 0;
    rfm_status rc = mlp_nparams(net, &np);
    if (rc != RFM_OK) return rc;
    rc = mlp_workspace(net, &wb);
    if (rc != RFM_OK) return rc;
    if (n_params) *n_params = np;
    if (ws_bytes) *ws_bytes = wb;
    return RFM_OK;
    RFM_GUARD_END
}

rfm_status rfm_mlp_forward(const rfm_mlp *net, const float *d_theta, const float *d_x, int64_t n, float *d_y,
                           void *stream) {
    RFM_GUARD_BEGIN
    if (!d_theta || (n > 0 && (!d_x || !d_y)) || n < 0) {
        set_error("rfm_mlp_forward: null argument or negative n");
        return RFM_EINVAL;
    }
    return launch_mlp_forward(net, d_theta, d_x, n, d_y, (cudaStream_t)stream);
    RFM_GUARD_END
}

rfm_status rfm_mlp_grad(const rfm_mlp *net, const float *d_theta, const float *d_x, const float *d_t, int64_t n,
                        float *d_grad, float *d_loss, void *d_ws, size_t ws_bytes, void *stream) {
    RFM_GUARD_BEGIN
    if (!d_theta || !d_x || !d_t || !d_grad) {
        set_error("rfm_mlp_grad: null argument");
        return RFM_EINVAL;
    }
    return launch_mlp_grad(net, d_theta, d_x, d_t, n, d_grad, d_loss, d_ws, ws_bytes, (cudaStream_t)stream);
    RFM_GUARD_END
}

rfm_status rfm_mlp_train_size(const rfm_mlp *net, int batch, size_t *ws_bytes) {
    RFM_GUARD_BEGIN
    if (!ws_bytes) {
        set_error("rfm_mlp_train_size: ws_bytes is NULL");
        return RFM_EINVAL;
    }
    return mlp_train_size(net, batch, ws_bytes);
    RFM_GUARD_END
}

rfm_status rfm_mlp_train(const rfm_mlp *net, float *d_theta, float *d_m, float *d_v, const float *d_x,
                         const float *d_t, const int64_t *d_order, int batch, int n_steps, int t0, const float *lr,
                         float beta1, float beta2, float eps, float *d_loss, void *d_ws, size_t ws_bytes,
                         void *stream) {
    RFM_GUARD_BEGIN
    if (!d_theta || !d_m || !d_v || !d_x || !d_t || !d_order || (n_steps > 0 && !lr)) {
        set_error("rfm_mlp_train: null argument");
        return RFM_EINVAL;
    }
    return launch_mlp_train(net, d_theta, d_m, d_v, d_x, d_t, d_order, batch, n_steps, t0, lr, beta1, beta2, eps,
                            d_loss, d_ws, ws_bytes, (cudaStream_t)stream);
    RFM_GUARD_END
}

rfm_status rfm_adam_step(int64_t n, float *d_theta, float *d_m, float *d_v, const float *d_g, int t, float lr,
                         float beta1, float beta2, float eps, void *stream) {
    RFM_GUARD_BEGIN
    if (!d_theta || !d_m || !d_v || !d_g) {
        set_error("rfm_adam_step: null argument");
        return RFM_EINVAL;
    }
    return launch_adam(n, d_theta, d_m, d_v, d_g, t, lr, beta1, beta2, eps, (cudaStream_t)stream);
    RFM_GUARD_END
}

}  // extern "C"
