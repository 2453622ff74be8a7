/*
 * rfm.h -- C ABI of the GB300 (sm_103a) library for ELM-FBPINNs with local
 * RRQR filtering and right preconditioning (van Beek, Dolean, Moseley, "Local
 * Feature Filtering for Scalable and Well-Conditioned Domain-Decomposed Random
 * Feature Methods").
 *
 * The path has four calls that follow the paper's problem statement:
 *   rfm_assemble     the block-sparse least-squares system M a = h of
 *                    Sec. 2.1 (Eqs. (1)-(5)) in the block form of Eq. (6);
 *   rfm_rrqr_filter  Algorithm 1: per block, Householder QR with column
 *                    pivoting stopped at |R_kk| < tol |R_11| (Sec. 3.1), and
 *                    the preconditioner factors of Sec. 3.2;
 *   rfm_lsqr_solve   Algorithm 2: LSQR (Paige and Saunders 1982) on the
 *                    right-preconditioned system M_hat S^-1 y = h, then
 *                    a = S^-1 y with zeros at dropped columns;
 *   rfm_eval         the ansatz of Eq. (1) at query points and the error
 *                    measures of Sec. 4.2.
 *
 * Conventions for every call:
 *  - All device memory belongs to the caller.  A system (one or more problem
 *    instances solved side by side) lives in one caller-allocated device
 *    workspace of rfm_problem_size()'s workspace_bytes; the library carves
 *    it and keeps nothing between calls.  The same instance list, count and
 *    rfm_config must be passed to every call on a workspace.
 *  - Calls are asynchronous on the given CUDA stream (NULL = legacy default
 *    stream): results are valid once the stream has reached the call.  No
 *    call allocates device memory or runs numerics on the host.  Host-side
 *    work is limited to O(J + grid size) layout bookkeeping.  Two calls
 *    upload small host tables with cudaMemcpyAsync from pageable host memory:
 *    rfm_assemble (instance and block records, work lists) and
 *    rfm_eval_noalloc (instance records).  CUDA may wait for the stream's
 *    earlier work before it stages such a copy, so these two calls can block
 *    the host until the stream reaches them; no other call of the path
 *    waits on the device (the QR autotuner and rfm_profile_read, which do,
 *    say so below).
 *  - Every call returns an rfm_status; on failure rfm_last_error() (per host
 *    thread) describes it.  No C++ exception crosses the ABI.
 *  - Device pointers must be aligned to 16 bytes and the workspace to 256.
 */
#ifndef RFM_H
#define RFM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RFM_ABI_VERSION 2

typedef enum {
    RFM_OK = 0,
    RFM_EINVAL = 1,     /* bad argument or problem description */
    RFM_ECUDA = 2,      /* a CUDA runtime call failed (message in rfm_last_error) */
    RFM_ENUMERIC = 3,   /* NaN/Inf met in a recurrence scalar */
    RFM_ETIMEOUT = 4,   /* a bounded device-side wait gave up (see rfm_lsqr_opts.timeout_ms) */
    RFM_ENOSPACE = 5    /* workspace smaller than rfm_problem_size() asks for */
} rfm_status;

/* PDE kinds: RFM_PDE_POISSON is -Laplace(u) = f with Dirichlet data on every
 * face; RFM_PDE_HEAT is u_t - kappa Laplace_x(u) = f where the last coordinate
 * is time, with Dirichlet data on the spatial faces (boundary set 0) and
 * initial data on t = lo (boundary set 1); RFM_PDE_OSC is the damped
 * oscillator of Sec. 4.1, m u'' + mu u' + k u = f in one dimension (time),
 * with (m, mu, k) = fam[0..2], the value u(lo) (boundary set 0) and the first
 * derivative u'(lo) (boundary set 1) given at the initial time, one row each. */
enum { RFM_PDE_POISSON = 0, RFM_PDE_HEAT = 1, RFM_PDE_OSC = 2 };

/* Activation Xi of every layer of the subdomain networks (Eq. (2); Tables 1
 * and 2 compare tanh with sigmoid and sine). */
enum { RFM_ACT_TANH = 0, RFM_ACT_SIGMOID = 1, RFM_ACT_SIN = 2 };

/* Manufactured data families (fam[] layout):
 *  RFM_FAM_SINPROD       u = sum_m fam[4m] prod_i sin(fam[4m+1+i] pi x_i);
 *                        f = -Laplace u, g = u.
 *  RFM_FAM_HEAT_SINPROD  u = sum_m fam[4m] exp(-kappa pi^2 |k_m|^2 t)
 *                        prod_{spatial i} sin(fam[4m+1+i] pi x_i); f = 0, g = u.
 *  RFM_FAM_PARAM5        f = sin(a pi x) sin(b pi y) + c sin(d pi x + e pi y),
 *                        g = 0 with (a,b,c,d,e) = fam[0..4]; no closed form.
 *  RFM_FAM_OSC           the under-damped oscillator (RFM_PDE_OSC) with
 *                        u(lo) = 1, u'(lo) = 0, f = 0: u = e^{-d s} (cos(w s)
 *                        + (d/w) sin(w s)), s = t - lo, d = mu/(2m),
 *                        w = sqrt(k/m - d^2). */
enum { RFM_FAM_SINPROD = 0, RFM_FAM_HEAT_SINPROD = 1, RFM_FAM_PARAM5 = 2, RFM_FAM_OSC = 3 };

/* One problem instance (Sec. 2.1 and the common settings of Sec. 4.2).
 *  dim            1..3; the box is prod_i [lo[i], hi[i]].
 *  S[i]           subdomains along dimension i (>= 2); J = prod S[i],
 *                 numbered lexicographically with dimension 0 fastest.
 *  delta          overlap ratio of Sec. 4.2 (subdomain width / centre
 *                 spacing): centre lo + (hi-lo) j/(S-1), half-width
 *                 (hi-lo) delta / (2 (S-1)).
 *  K              random tanh features per subdomain.
 *  n[i]           cell-centred interior collocation points per dimension;
 *                 boundary rows sit on each face at the interior grid of the
 *                 other dimensions.  Row order: interior (dimension 0
 *                 fastest), then faces (dim 0 lo, dim 0 hi, dim 1 lo, ...).
 *  lam[l]         loss weight of boundary set l (Eq. (3)).
 *  family, n_modes, fam[]: the data, see above.
 *  depth          h of Eq. (2), 1..8 (0 reads as 1): h - 1 hidden layers of
 *                 K units (K <= 32 when h > 1) before the K features.
 *  act            RFM_ACT_*, the activation of every layer.
 *  hard_bc        0, or c > 0: the hard-constraint ansatz of the Laplace
 *                 problem (Sec. 4.1), u = g(x) u_hat(x) with g = prod_i
 *                 tanh(c (x_i - lo_i)) tanh(c (hi_i - x_i)); the instance then
 *                 has no boundary rows (Poisson only).
 * Network parameters of one subdomain (the d_params layout): the output
 * layer first, one row (w_1 .. w_n, b) per feature with n = dim for h = 1 and
 * n = K otherwise, then every hidden layer l = 1 .. h-1 as its weights (K x
 * n_{l-1}, row-major, n_0 = dim) followed by its biases (K).  A feature is
 * Xi(w . z + b) with z the normalised coordinates (x - mu)/sig for h = 1, or
 * the last hidden layer's output. */
typedef struct rfm_problem {
    int32_t dim, pde, family, n_modes;
    int32_t S[3], n[3];
    int32_t K, reserved0;
    double delta, kappa;
    double lo[3], hi[3];
    double lam[2];
    double fam[64];
    int32_t depth, act;
    double hard_bc;
} rfm_problem;

/* Arithmetic of the assembly. */
enum { RFM_ASM_FP64 = 0, RFM_ASM_FP32 = 1 };

/* LSQR operator (all are the same preconditioned operator of Algorithm 2 up
 * to rounding, except RFM_OP_PLAIN):
 *  RFM_OP_AR64    M_hat S^-1 applied as the FP64 kept columns followed by
 *                 FP64 substitution with R_hat_j (Sec. 3.2).
 *  RFM_OP_Q32     the explicit orthonormal blocks Q_hat_j of Proposition 3.1,
 *                 formed in FP64 from the reflectors and stored in FP32;
 *                 FP32 products with FP32 accumulation, FP64 vectors and
 *                 scalars (mixed precision).
 *  RFM_OP_Q64     Q_hat_j kept in FP64.
 *  RFM_OP_PLAIN   the unfiltered, unpreconditioned M in FP64 (the paper's
 *                 plain-LSQR baseline of Sec. 4.3); the filter call then only
 *                 records the blocks. */
enum { RFM_OP_AR64 = 0, RFM_OP_Q32 = 1, RFM_OP_Q64 = 2, RFM_OP_PLAIN = 3 };

typedef struct rfm_config {
    int32_t asm_prec;   /* RFM_ASM_FP64 or RFM_ASM_FP32 */
    int32_t op;         /* RFM_OP_* */
    double tol;         /* relative drop threshold sigma of Algorithm 1 */
} rfm_config;

/* Sizes of a system (sums over its instances). */
typedef struct rfm_sizes {
    int64_t n_inst;
    int64_t n_blocks;        /* sum of J over instances */
    int64_t n_rows;          /* sum of N = N_I + N_B */
    int64_t n_cols;          /* sum of J K (the layout of a and y) */
    int64_t block_rows;      /* sum over blocks of |I_j| rounded up to a multiple of 32
                                (block rows are laid out at that padded stride) */
    int64_t max_block_rows;  /* max |I_j| */
    int64_t max_K;
    int64_t workspace_bytes; /* device bytes the caller must provide */
} rfm_sizes;

/* Host only.  Validates the instances and computes the system's sizes.
 * Errors: RFM_EINVAL for an invalid instance (dim outside 1..3, S < 2, K < 1
 * or > 1024, n < 1, delta <= 0, a subdomain with no collocation point, a
 * block taller than 4194304 rows, depth outside 0..8, depth > 1 with K > 32,
 * an unknown activation, a negative hard_bc or one on a non-Poisson instance,
 * or RFM_PDE_OSC other than in one dimension with RFM_FAM_OSC). */
rfm_status rfm_problem_size(const rfm_problem *probs, int n_inst, const rfm_config *cfg, rfm_sizes *out);

/* Assembly (Sec. 2.1, Eqs. (1)-(6)).  For every block j the dense local
 * matrix M_j = M restricted to I_j x K_j, with I_j = {r : w_j(x_r) != 0}:
 * interior rows N[w_j phi_jk](x)/sqrt(N_I), boundary rows
 * sqrt(lam_l/N_B^(l)) w_j phi_jk(x), and h = [f/sqrt(N_I); sqrt(lam_l/N_B^(l)) g].
 * Features phi_jk of Eq. (2) (for h = 1, phi_jk = Xi(sum_i w_i (x_i -
 * mu_i)/sig_i + b)) with the parameters read from d_params: per instance J
 * subdomain networks in the layout described at rfm_problem (for h = 1:
 * J*K*(dim+1) doubles, (j, k, [w_1..w_d, b]) row-major), instances
 * concatenated in order.  Windows: the normalised cosine window of Sec. 4.2,
 * times the hard-constraint factor g when hard_bc > 0 (the operator then acts
 * on g w_j phi_jk).  Writes the workspace only. */
rfm_status rfm_assemble(const rfm_problem *probs, int n_inst, const rfm_config *cfg, const double *d_params,
                        void *d_ws, size_t ws_bytes, void *stream);

/* Filtering and preconditioner factors (Algorithm 1, Sec. 3.1-3.2).  Per
 * block: Householder QR with column pivoting in FP64 (pivot = largest
 * trailing column norm, norms downdated in FP64 with recomputation when
 * cancellation makes the downdate unreliable; ties to the lowest original
 * index), stopped at the first step whose |R_kk| is zero or below
 * cfg->tol * |R_11|.  Keeps r_j columns; then prepares the operator that
 * cfg->op names (kept columns, or Q_hat_j from the reflectors).
 * d_rank (nullable, n_blocks int32) receives r_j; d_perm (nullable,
 * n_blocks*K int32) the pivoted column order (first r_j entries = kept). */
rfm_status rfm_rrqr_filter(const rfm_problem *probs, int n_inst, const rfm_config *cfg, void *d_ws, size_t ws_bytes,
                           int32_t *d_rank, int32_t *d_perm, void *stream);

typedef struct rfm_lsqr_opts {
    double atol, btol;   /* stopping tolerances of Paige and Saunders (0 = run max_iter) */
    int32_t max_iter;
    int32_t timeout_ms;  /* bound on every device-side wait; 0 = 10000 */
    double *d_snap;      /* nullable: iterate snapshots, snap_cap x n_cols doubles; after
                            iteration i = s*snap_every (s = 1..snap_cap) y_i is written to
                            row s-1 (kept slots only; the caller clears the buffer) */
    int32_t snap_every, snap_cap;
    double *d_phase_ms;  /* nullable, 4 doubles: milliseconds the first CTA spent in each
                            part of the iterations (fused products A^T u and A x with the
                            column updates; row sums with the scalar updates overlapped; 0;
                            0), each up to the exit of the grid barrier that closes it; for
                            profiling; not written with RFM_OP_AR64 */
    int32_t refine_steps;  /* iterative refinement: correction solves after the first solve
                              (0..64; 0 = none), see rfm_lsqr_solve */
    int32_t refine_iters;  /* iteration limit of each correction solve (0 = max_iter) */
    double *d_rnorm64;     /* nullable: n_inst x (refine_steps + 1) doubles (row-major), the
                              residual ||h - M a_s|| of the assembled system evaluated in FP64
                              after solve s = 0 .. refine_steps */
} rfm_lsqr_opts;

/* Report per instance (written to device memory):
 *   itn, istop (0 exact start, 1 residual test, 2 normal-equation test,
 *   7 iteration limit), rnorm, arnorm, anorm, ynorm, bnorm estimates,
 *   status (an rfm_status of the device-side run),
 *   start: 1 when the warm start y0 was used, 0 for a zero start (no y0, or
 *   a y0 whose residual ||h - A S^-1 y0|| was not below ||h||, the fallback),
 *   r0norm: ||h - A S^-1 y0|| of the given y0 (||h|| without y0).
 * With refinement, itn counts the iterations of every solve and the other
 * estimates are those of the last correction solve (on its own right-hand
 * side); d_rnorm64 carries the residuals of the assembled system. */
typedef struct rfm_lsqr_report {
    double itn, istop, rnorm, arnorm, anorm, ynorm, bnorm, status;
    double start, r0norm;
} rfm_lsqr_report;

/* LSQR on min ||M_hat S^-1 y - h|| for every instance at once (each with its
 * own scalars and stopping test), then a = S^-1 y scattered to the J*K layout
 * with zeros at dropped columns (Algorithm 2).
 *  d_y0     nullable warm start (n_cols doubles, per block the first r_j of
 *           each K-slot used); the iteration runs on the residual system.
 *           Per instance, a y0 whose residual ||h - A S^-1 y0|| is not below
 *           ||h|| is dropped for a zero start (report field start = 0).
 *  d_y      nullable output y (n_cols doubles, same layout; 0 at dropped slots).
 *  d_a      output coefficients (n_cols doubles).
 *  d_report n_inst rfm_lsqr_report.
 * Stopping (per instance): ||r|| <= btol ||h|| + atol ||A||_F ||y||, or
 * ||A^T r|| <= atol ||A||_F ||r||, or max_iter, with the norm estimates of
 * the 1982 paper and ||y|| computed exactly.
 * Iterative refinement (opts->refine_steps = R > 0; the paper solves once,
 * this is the mixed-precision refinement of Carson and Higham, "Accelerating
 * the solution of linear systems by iterative refinement in three
 * precisions", SISC 2018, applied to the least-squares problem of
 * Algorithm 2): after the first solve, R times: a = S^-1 y, the residual
 * r = h - M a of the assembled system in FP64 (FP64 blocks, or the FP32
 * blocks' values taken exactly), a correction solve min ||M_hat S^-1 d - r||
 * from zero with the configured operator (at most refine_iters iterations,
 * same atol and btol), y += d.  With an FP32 operator this brings the mixed
 * path to the FP64 least-squares solution of the kept columns.  The h and M
 * arenas are read, not changed.
 * The call is asynchronous: a device-side wait (grid barrier or the wait of
 * a forward tile on its block) that runs longer than timeout_ms ends the
 * kernel at that wait, and every report's status is then RFM_ETIMEOUT
 * (results invalid); a non-finite recurrence gives RFM_ENUMERIC there.
 * Errors: RFM_EINVAL for more than 64 instances, refine_steps outside 0..64
 * or a negative refine_iters. */
rfm_status rfm_lsqr_solve(const rfm_problem *probs, int n_inst, const rfm_config *cfg, const rfm_lsqr_opts *opts,
                          const double *d_y0, double *d_y, double *d_a, rfm_lsqr_report *d_report,
                          void *d_ws, size_t ws_bytes, void *stream);

/* Residual of the assembled least-squares system (Eqs. (4)-(5)) at
 * coefficients d_a (n_cols doubles, the J*K layout of rfm_lsqr_solve):
 * r = h - M a in FP64 from the stored blocks (FP64, or the FP32 blocks'
 * values taken exactly), each row summed over its blocks in a fixed order.
 * d_r (nullable, n_rows doubles) receives r; d_rnorm (nullable, n_inst
 * doubles) ||r|| per instance.  Uses the workspace's row scratch (do not
 * overlap with rfm_lsqr_solve on the same workspace).  Requires rfm_assemble. */
rfm_status rfm_residual(const rfm_problem *probs, int n_inst, const rfm_config *cfg, const double *d_a, double *d_r,
                        double *d_rnorm, void *d_ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Many right-hand sides on one operator.  Data sets of one family that share
 * the decomposition, the features and the collocation (every field of
 * rfm_problem but family, n_modes and fam; the oscillator's coefficients
 * fam[0..2] included) share M, so Algorithm 1's factors and Proposition 3.1's
 * Q_hat_j are those of one system; only h differs.  LSQR then runs for every
 * data set at once, each with its own scalars, estimates and stopping test,
 * and the block products of an iteration read Q_hat_j once for all of them:
 * dense (m_j x r_j) x (r_j x nrhs) products.  The paper solves one data set
 * at a time; this is an implementation choice.
 * ------------------------------------------------------------------------ */

/* Bytes of the multi-right-hand-side workspace for nrhs data sets (1..256)
 * of the system described by prob (one instance). */
rfm_status rfm_lsqr_multi_size(const rfm_problem *prob, const rfm_config *cfg, int nrhs, size_t *bytes);

/* h (Eq. (5)) of data sets probs[0..nrhs) into d_H (nrhs x n_rows doubles,
 * set j at d_H + j n_rows).  Every probs[j] must equal probs[0] except in its
 * data (RFM_EINVAL otherwise).  d_mws: the multi-right-hand-side workspace
 * (rfm_lsqr_multi_size bytes, 256-byte aligned); its first bytes receive the
 * sets' records, uploaded with cudaMemcpyAsync from pageable host memory. */
rfm_status rfm_rhs_many(const rfm_problem *probs, int nrhs, const rfm_config *cfg, double *d_H, void *d_mws,
                        size_t mws_bytes, void *stream);

/* LSQR of Algorithm 2 for nrhs right-hand sides d_H (layout of
 * rfm_rhs_many) on the filtered system in d_ws (assembled and filtered with
 * RFM_OP_Q32 or RFM_OP_Q64, one instance), then a_j = S^-1 y_j into d_A
 * (nrhs x n_cols doubles, set j at d_A + j n_cols, zeros at dropped
 * columns), d_report[j] per set.  opts: atol, btol, max_iter (the other
 * fields unused).  d_Y0: nullable warm starts, nrhs x n_cols doubles in the
 * y layout of rfm_lsqr_solve's d_y0 (set j at d_Y0 + j n_cols); as there, a
 * set keeps its start only when ||h_j - A S^-1 y0_j|| < ||h_j|| and falls
 * back to zero otherwise (report fields start, r0norm).  Without d_Y0 every
 * set starts from zero.  Every set stops on the tests of rfm_lsqr_solve, with
 * ||y|| of the previous iteration.  The call issues a fixed sequence of
 * launches per iteration (max_iter of them, without waiting on the host;
 * sets that have stopped keep their iterate, and once every set has stopped
 * the block products and vector passes of the remaining iterations return at
 * once) and uploads its tile lists from pageable host memory.
 * Errors: RFM_EINVAL for another operator, more than one instance, nrhs
 * outside 1..256 or bad options; RFM_ENOSPACE for a short workspace. */
rfm_status rfm_lsqr_multi(const rfm_problem *prob, const rfm_config *cfg, const rfm_lsqr_opts *opts, int nrhs,
                          const double *d_H, const double *d_Y0, double *d_A, rfm_lsqr_report *d_report, void *d_ws,
                          size_t ws_bytes, void *d_mws, size_t mws_bytes, void *stream);

/* a = S^-1 y (Algorithm 2's last step) for an arbitrary y in the n_cols
 * layout: per block a_j[perm[c]] = (R_hat_j^-1 y_j)[c] for kept c, 0 at
 * dropped columns (RFM_OP_PLAIN: a = y).  Requires a filtered workspace. */
rfm_status rfm_coefficients(const rfm_problem *probs, int n_inst, const rfm_config *cfg, const double *d_y,
                            double *d_a, void *d_ws, size_t ws_bytes, void *stream);

/* Ansatz of Eq. (1), u_hat(x) = sum_j w_j(x) sum_k a_jk phi_jk(x), in FP64 at
 * query points, and error sums against the family's closed-form u.
 *  d_x      points, 3 doubles each (unused coordinates ignored), instances
 *           concatenated; h_pt_off host array of n_inst+1 offsets.
 *  d_u      output u_hat per point.
 *  d_err    nullable, 4 doubles per instance: sum (u_hat-u)^2, sum u^2,
 *           sum |u_hat-u|, sum u (relative L2 and e_L1 of Sec. 4.2 follow).
 * Uses the workspace (it must have been assembled) for its reduction scratch. */
rfm_status rfm_eval(const rfm_problem *probs, int n_inst, const rfm_config *cfg, const double *d_params,
                    const double *d_a, const double *d_x, const int64_t *h_pt_off, double *d_u, double *d_err,
                    void *d_ws, size_t ws_bytes, void *stream);

/* Allocation-free variant of rfm_eval (the paper has no counterpart; this is
 * a deployment convenience).  For callers that cannot allocate device memory
 * or hold a workspace -- code running inside another framework's memory pool,
 * plugin hosts that only pass in input and output buffers, processes whose
 * device memory is reserved up front.  Same arguments and results as
 * rfm_eval, without a workspace: the instance records and the per-CTA error
 * partials live in a static device array of about 0.5 MB that every GPU
 * loading this library holds until the process exits.
 *  - At most 16 instances per call (more: RFM_EINVAL with a message).
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  Later calls may be captured into a CUDA
 *    graph: the instance records travel as kernel parameters (no copy from
 *    host memory), so a replay evaluates the captured problems at the
 *    current contents of the captured device buffers.
 *  - The call allocates no device memory and calls no allocating library
 *    routine.  Every call shares the array, which keeps the last call's
 *    contents; each call overwrites what it reads, so nothing needs clearing,
 *    but calls that overlap on the GPU (different streams, or several host
 *    threads) race on the array: serialise them. */
rfm_status rfm_eval_noalloc(const rfm_problem *probs, int n_inst, const double *d_params, const double *d_a,
                            const double *d_x, const int64_t *h_pt_off, double *d_u, double *d_err, void *stream);

/* ------------------------------------------------------------------------
 * Learned warm start.  The paper solves every problem from a zero start; these
 * calls add a starting point predicted by a small network trained on earlier
 * solutions (a method extension with no counterpart in the paper).  The
 * prediction u_hat at every block's rows is fitted, block by block, through
 * the block's kept features, and the fitted coefficients c_j become the LSQR
 * starting point y0_j = R_j c_j of Algorithm 2's preconditioned unknowns
 * (pass it as y0 to rfm_lsqr_solve).  The stopping rule of the solve is
 * unchanged, so a zero start remains the fallback and the yardstick for the gain.
 * ------------------------------------------------------------------------ */

/* Network inputs at every block row (rows in the block-row layout of
 * rfm_block_info: block b's rows at roff .. roff + ldm, padding rows zero):
 * d_x[row, :] = [ctx of the row's instance (n_ctx floats, from d_ctx, n_inst x
 * n_ctx row-major), centre of the block (dim), (x - centre) / half-width
 * (dim)], FP32, row-major with n_ctx + 2 dim columns.  d_pts (optional, may be
 * NULL) receives the row's point (3 doubles per row, unused coordinates 0).
 * Needs the records written by rfm_assemble. */
rfm_status rfm_block_inputs(const rfm_problem *probs, int n_inst, const rfm_config *cfg, const float *d_ctx,
                            int n_ctx, float *d_x, double *d_pts, void *d_ws, size_t ws_bytes, void *stream);

/* Bytes of the fit workspace of a system (three FP64 block arenas of the
 * system's block shape plus per-column pivots). */
rfm_status rfm_fit_size(const rfm_problem *probs, int n_inst, const rfm_config *cfg, size_t *bytes);

/* Per block: the window-weighted values of the kept features (pivot order of
 * rfm_rrqr_filter) at the block's rows, factored by QR with column pivoting
 * truncated at tol_fit |R_11| (the same kernels as Algorithm 1), with explicit
 * Q_hat.
 * Needs rfm_assemble and rfm_rrqr_filter on d_ws (any operator but PLAIN).
 * Instances with one-layer tanh networks only (RFM_EINVAL otherwise).
 * d_fit_ws: 256-byte aligned, rfm_fit_size bytes, owned by the caller. */
rfm_status rfm_fit_prepare(const rfm_problem *probs, int n_inst, const rfm_config *cfg, const double *d_params,
                           double tol_fit, void *d_ws, size_t ws_bytes, void *d_fit_ws, size_t fit_bytes,
                           void *stream);

/* y0 from predictions d_uhat (FP32, block-row layout as rfm_block_inputs),
 * multiplied per instance by d_inst_scale[inst] when that is not NULL (a
 * network trained on targets brought to a common scale).
 * fit_iters = 0: local fit, per block the truncated least-squares coefficients
 * c_j of w_j u_hat_j in the window-weighted kept features.  fit_iters > 0:
 * global fit, the blended prediction sum_j w_j u_hat_j at every collocation
 * row fitted through all blocks' window-weighted kept features at once by
 * fit_iters LSQR iterations on the block-preconditioned fitting system (the
 * system's LSQR scratch is reused: do not overlap with rfm_lsqr_solve on the
 * same workspace).  Then y0 = R_j c_j in the column-slot layout of
 * rfm_lsqr_solve (slots beyond a block's rank set to 0). */
rfm_status rfm_warm_start(const rfm_problem *probs, int n_inst, const rfm_config *cfg, const float *d_uhat,
                          const float *d_inst_scale, int fit_iters, double *d_y0, void *d_ws, size_t ws_bytes,
                          void *d_fit_ws, size_t fit_bytes, void *stream);

/* The network: fully connected, widths width[0..n_layers], tanh on hidden
 * layers, one linear output (width[n_layers] = 1); input width 1..32, hidden
 * widths multiples of 16 up to 128, at most 8 layers.  Parameters FP32, packed
 * layer by layer: W_l row-major (width[l] x width[l-1]) then b_l. */
typedef struct {
    int32_t n_layers;
    int32_t width[9];
} rfm_mlp;

/* Parameter count and the workspace bytes of rfm_mlp_grad (any batch size). */
rfm_status rfm_mlp_size(const rfm_mlp *net, int64_t *n_params, size_t *ws_bytes);

/* d_y[i] = network(d_x[i, :]) for n samples (d_x row-major n x width[0]).
 * On the tensor-core path (RFM_OPT_MLP_TENSOR_CORES) a wait for the MMAs
 * that runs out (about a second) leaves NaN in the CTA's outputs. */
rfm_status rfm_mlp_forward(const rfm_mlp *net, const float *d_theta, const float *d_x, int64_t n, float *d_y,
                           void *stream);

/* Mean squared error (1/n) sum_i (network(x_i) - t_i)^2 over the batch and its
 * gradient (n_params floats) by backpropagation; d_loss (1 float, may be
 * NULL).  The per-CTA partial gradients are summed in a fixed order, so the
 * result is reproducible on a given GPU.  On the tensor-core path a wait for
 * the MMAs that runs out leaves NaN in the gradient and the loss. */
rfm_status rfm_mlp_grad(const rfm_mlp *net, const float *d_theta, const float *d_x, const float *d_t, int64_t n,
                        float *d_grad, float *d_loss, void *d_ws, size_t ws_bytes, void *stream);

/* One Adam step (Kingma and Ba 2015) at step number t >= 1 on n parameters:
 * moments d_m, d_v and parameters updated in place from gradient d_g. */
rfm_status rfm_adam_step(int64_t n, float *d_theta, float *d_m, float *d_v, const float *d_g, int t, float lr,
                         float beta1, float beta2, float eps, void *stream);

/* Minibatch training loop on the host side of the library: n_steps steps,
 * step k gathering the batch d_x[d_order[k batch + s], :], d_t[...] (s <
 * batch; d_order: device int64, n_steps * batch sample indices, each < the
 * caller's sample count), then rfm_mlp_grad on it and rfm_adam_step with step
 * number t0 + k and learning rate lr[k] (host array of n_steps floats).
 * d_loss (device, n_steps floats, may be NULL) receives each step's batch
 * loss.  Parameters and moments are updated in place, exactly as the
 * separate calls would, without a host round trip between the steps'
 * launches.  d_ws: 256-byte aligned, rfm_mlp_train_size bytes for this batch
 * size.  Not in the paper: the training of the warm-start network. */
rfm_status rfm_mlp_train_size(const rfm_mlp *net, int batch, size_t *ws_bytes);
rfm_status rfm_mlp_train(const rfm_mlp *net, float *d_theta, float *d_m, float *d_v, const float *d_x,
                         const float *d_t, const int64_t *d_order, int batch, int n_steps, int t0, const float *lr,
                         float beta1, float beta2, float eps, float *d_loss, void *d_ws, size_t ws_bytes,
                         void *stream);

/* Device-side copies of the assembled blocks for inspection and tests:
 * block b's M_j (|I_j| x K, column-major with leading dimension *ld) starts at
 * element offset *moff of the M arena, and its rows are the global rows
 * grow[roff .. roff+|I_j|).  Host only. */
rfm_status rfm_block_info(const rfm_problem *probs, int n_inst, const rfm_config *cfg, int64_t block,
                          int64_t *m, int64_t *ld, int64_t *moff, int64_t *roff);

/* The global rows (across instances) of block b's rows I_j (Eq. (6)), in
 * the block's row order: interior rows, then its face rows (host array of
 * |I_j| entries).  Host only; the partition of a system over several
 * processes is built from it. */
rfm_status rfm_block_rows(const rfm_problem *probs, int n_inst, const rfm_config *cfg, int64_t block,
                          int64_t *rows);

/* rfm_block_info for every block at once: host arrays of n_blocks entries
 * (any may be NULL). */
rfm_status rfm_block_table(const rfm_problem *probs, int n_inst, const rfm_config *cfg, int64_t *m, int64_t *ld,
                           int64_t *moff, int64_t *roff);

/* The order in which the filter's QR clusters take the blocks (n_blocks
 * indices, host array): decreasing m K min(m, K), the leading term of the
 * block's factorization flops, ties by block index.  A scheduling choice of
 * this implementation (row a7 of the batched workload); the paper has no
 * counterpart.  Host only. */
rfm_status rfm_qr_order(const rfm_problem *probs, int n_inst, const rfm_config *cfg, int32_t *order);

/* Device pointers into the workspace (views for tests and for the warm
 * start): which = 0 M arena (FP64 or FP32 by asm_prec), 1 h (FP64, n_rows),
 * 2 grow (int32, block_rows; global row index across instances),
 * 3 QR work (FP64, R above the diagonal, reflectors below), 4 r11 (FP64 per
 * block), 5 operator arena (Q32: FP32; others FP64). */
rfm_status rfm_workspace_view(const rfm_problem *probs, int n_inst, const rfm_config *cfg, void *d_ws, int which,
                              void **ptr);

/* Kernel timing for profiling (process-wide, host side).  While enabled,
 * every kernel the library launches is bracketed by CUDA events on its
 * stream.  rfm_profile_read waits for the recorded events and returns up to
 * max entries (name, launches, total milliseconds) aggregated by kernel name
 * since the last reset; the return value is the number of entries.  Events
 * are created with cudaEventCreate (no device memory).  Not for use inside
 * stream capture. */
rfm_status rfm_profile_enable(int on);
rfm_status rfm_profile_reset(void);
int rfm_profile_read(const char **names, int64_t *launches, double *ms, int max);

/* Process-wide options (host side).
 *  RFM_OPT_FILTER_KERNEL: 0 (default) chooses per system: the cluster kernel
 *    (block held in the distributed shared memory of a cluster of up to 8
 *    CTAs) when the largest block fits, else the global-memory kernel;
 *    1 forces the global-memory kernel (for comparison and testing).
 *  RFM_OPT_AUTOTUNE: 1 makes the first rfm_rrqr_filter (and rfm_fit_prepare)
 *    call for a block shape (largest block rows and features, assembly
 *    precision, block count) time every cluster size the blocks fit -- or,
 *    for blocks too large for a cluster, 8, 16 and 32 warps per block of the
 *    global-memory kernels, then the panel widths of RFM_OPT_QR_PANEL that
 *    fit -- and keep the fastest for later calls in the
 *    process; that first call waits for its own timing runs (it synchronises
 *    the stream).  0 (default) takes the smallest cluster that holds the
 *    largest block, or RFM_OPT_QR_WARPS warps.
 *  RFM_OPT_QR_DOUBLE_FLOAT: 1 (default) factors FP32-assembled blocks in the
 *    cluster kernel with double-float arithmetic (pairs of FP32 numbers, about
 *    48 significant bits, on the FP32 pipe; the reflector scalars, norms fed
 *    to the threshold test and R are formed in FP64) unless Q_hat is wanted in
 *    FP64; 0 uses FP64 arithmetic for them too.  2 also factors FP64-assembled
 *    blocks in double-float when the operator is RFM_OP_Q32 (each FP64 entry
 *    split into two FP32 numbers on load, relative error 2^-48; the mixed
 *    path with refinement); with 0 or 1 FP64-assembled blocks use FP64
 *    arithmetic.
 *  RFM_OPT_LSQR_STALL (test hook for failure detection): 1 makes the first
 *    grid barrier of the next explicit-operator solves wait for an arrival
 *    that never comes, 2 makes their forward tiles wait for a chunk that never
 *    finishes; the bounded waits then run out after timeout_ms, the kernel
 *    leaves and the report's status is RFM_ETIMEOUT.  0 (default) is off.
 *  RFM_OPT_MLP_TENSOR_CORES: 1 (default) runs rfm_mlp_forward and
 *    rfm_mlp_grad on the tensor cores (tcgen05, BF16 operands, FP32
 *    accumulation) when every hidden layer is 128 wide (rfm_mlp_grad: one to
 *    three 128 x 128 layers and fewer than 32 inputs); results then carry
 *    BF16 rounding (about 1e-2 relative).  0 keeps the FP32 kernels for every
 *    network.
 *  RFM_OPT_QR_ORDER: 1 (default) starts the QR of the blocks with the most
 *    work (m K min(m, K), largest first), so that a batch of uneven blocks
 *    does not end on a few large ones; 0 takes them in block order.  The
 *    factors are the same either way.
 *  RFM_OPT_MLP_TC_THREADS: threads per CTA of the tensor-core network
 *    kernels, 512 (default: four threads per sample, each with 32 of the 128
 *    columns) or 256 (two per sample).  The results are the same.
 *  RFM_OPT_LSQR_LAG: how far (in tenths of one pass of the grid's warps over
 *    the work list, 1..100) a block's row tiles of the forward product follow
 *    its column chunks of the transposed product in the explicit-operator
 *    LSQR kernel; 0 (default) takes 1.6 passes, capped so that about 120 MB
 *    of operator lie in between.  Shorter lags keep the block in L2 for its
 *    second read, longer ones keep the tiles from waiting on the chunks; the
 *    iterates agree to rounding (the per-warp partial sums change).
 *  RFM_OPT_MULTI_TENSOR_CORES: 1 (default) forms rfm_lsqr_multi's block
 *    products of the FP32 operator on the tensor cores (tcgen05, every FP32
 *    operand split into three BF16 terms, six products accumulated in FP32:
 *    FP32-grade products); 0 on the CUDA cores in FP32.  The FP64 operator's
 *    products always run on the CUDA cores.  The iterates agree to rounding.
 *  RFM_OPT_QR_WARPS: warps per CTA (4, 8, 16 or 32 (default)) of the
 *    global-memory QR kernels (blocks too large for a cluster: one CTA per
 *    block, warps over the trailing columns).  The factors agree to rounding
 *    (the pivot column's norm is summed in another order).
 *  RFM_OPT_QR_PANEL: panel width of those kernels on FP32-assembled blocks in
 *    double-float arithmetic: 1 (one step at a time), 2, 4 or 8 (default),
 *    narrowed to what fits in shared memory.  The QR with column pivoting
 *    defers the trailing update over panels of up to 4 of its steps
 *    (Quintana-Orti, Sun and Bischof: per step one read of the trailing
 *    columns, the pivot row and the norm downdates; one rank-nb update per
 *    panel), and the FP32 Q_hat is formed from compact WY panels
 *    I - V T V^T of the full width.  With
 *    RFM_OPT_AUTOTUNE the first call for a block shape times every width
 *    that fits and keeps the fastest.  R and Q_hat agree to rounding; the
 *    kept columns agree except where two trailing norms tie to within it. */
enum {
    RFM_OPT_FILTER_KERNEL = 0,
    RFM_OPT_AUTOTUNE = 1,
    RFM_OPT_QR_DOUBLE_FLOAT = 2,
    RFM_OPT_LSQR_STALL = 3,
    RFM_OPT_MLP_TENSOR_CORES = 4,
    RFM_OPT_QR_ORDER = 5,
    RFM_OPT_MLP_TC_THREADS = 6,
    RFM_OPT_LSQR_LAG = 7,
    RFM_OPT_MULTI_TENSOR_CORES = 8,
    RFM_OPT_QR_WARPS = 9,
    RFM_OPT_QR_PANEL = 10
};
rfm_status rfm_set_option(int option, int value);

const char *rfm_last_error(void);
int rfm_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif
