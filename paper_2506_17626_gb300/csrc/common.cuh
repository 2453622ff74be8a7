// common.cuh -- layout records shared by the library's kernels and host code.
//
// A "system" is a list of problem instances solved side by side.  The host
// side (plan.cu) turns the instance descriptions into per-instance and
// per-block records plus small per-dimension index tables, places every array
// of the system inside the caller's workspace, and uploads the records once
// (rfm_assemble).  Kernels read the records from the workspace.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rfm.h"

namespace rfm {

constexpr int kMaxInst = 256;      // instances per system
constexpr int kMaxK = 1024;        // features per subdomain
constexpr int kLdAlign = 32;       // row padding of every block (128 B in FP32, 256 B in FP64)
constexpr int kMaxFaces = 6;
constexpr int kMaxPersistCtas = 2048;  // upper bound of the persistent LSQR grid

// Per-instance record (device copy in the workspace).
struct InstRec {
    int32_t dim, pde, family, n_modes;
    int32_t n[3], S[3];
    int32_t K, nfaces, C, blk0;
    int32_t nblk, pad0;
    int32_t maxcover[3];
    int32_t pad1;
    double lo[3], hi[3];
    double kappa, scale_int, scale_set[2];
    double delta, pad2;
    double fam[64];
    int64_t row0, N, NI;        // rows of this instance are row0 .. row0+N
    int64_t face_row0[kMaxFaces];  // instance-local row offset of each face (NI + preceding faces)
    int64_t col0;               // first column (J*K layout)
    int64_t rl_off;             // offset of this instance's row lists (C per row)
    int64_t prm_off;            // offset (doubles) of the instance's feature parameters
    int32_t cov_off[3];         // offset of per-dimension cover tables (n[i] + 2 entries)
    int32_t pad3;
    int32_t depth, act;         // subdomain networks (Eq. (2)): depth h >= 1, activation
    double hard_bc;             // factor of the hard-constraint ansatz (0: none)
    int64_t n_prm_sub;          // parameters of one subdomain network (doubles)
    int32_t n_last, pad4;       // inputs of the output layer: dim (h = 1) or K
};

constexpr int kMaxDeepK = 32;   // width limit of networks with hidden layers

// Normal dimension and side of face f (the oscillator's two initial rows both
// sit at the lower end of its one dimension).
__host__ __device__ inline void face_dims(int pde, int f, int *nd, int *side) {
    if (pde == RFM_PDE_OSC) {
        *nd = 0;
        *side = 0;
        return;
    }
    *nd = f / 2;
    *side = f % 2;
}

// Boundary set of face f: heat's initial face is set 1; the oscillator's
// value row set 0 and derivative row set 1; every other face set 0.
__host__ __device__ inline int face_set_of(int pde, int dim, int f) {
    if (pde == RFM_PDE_OSC) return f;
    return (pde == RFM_PDE_HEAT && f / 2 == dim - 1) ? 1 : 0;
}

// Per-block record: block b is subdomain j of instance inst.
struct BlkRec {
    int32_t inst, j, m, ldm;       // rows |I_j|, padded leading dimension
    int32_t K, n_int, pad0, pad1;  // features, interior rows
    int32_t jd[3], pad2;           // subdomain index per dimension
    int32_t box_lo[3], box_n[3];   // interior grid box of the block
    int32_t face_off[kMaxFaces];   // first block-local row of face f (-1: face not touched)
    int64_t moff;                  // element offset of the block in every (ldm x K) arena
    int64_t roff;                  // offset into block-row arrays
    int64_t coff;                  // offset of the block's K-slot in column vectors
    int64_t pad3;
    double mu[3], sig[3];
};

// A live column item of the LSQR kernels: columns c0 .. c0+nc of block b.
struct ColItem {
    int32_t b, c0, nc, m, ldm, inst;
    int64_t moff, coff, roff;
};

// Persistent LSQR scalars, one per instance.
struct LsqrScal {
    double alpha, beta, rhobar, phibar, anorm2, bnorm;
    double rnorm, arnorm, ynorm, phi_rho, theta_rho, c;
    double r0norm;              // ||h - Op y0|| of the given start (||h|| without one)
    int32_t itn, istop, done, status;
    int32_t start, pad;         // 1: the warm start is used, 0: zero start
};

// Offsets (bytes) of every array of a system inside the workspace.
struct Layout {
    int n_inst;
    int64_t n_blocks, n_rows, n_cols, block_rows, max_m, max_K, n_rowlist, n_tiles, n_cov;  // block_rows: padded
    size_t off_inst, off_blk, off_tile, off_cov;       // records
    size_t off_M, off_h, off_grow, off_rowlist;         // assembly
    size_t off_W, off_tau, off_perm, off_rank, off_r11, off_op, off_q32;  // filter
    size_t off_u, off_v, off_vt, off_w, off_y, off_t, off_part, off_scal, off_bar;  // lsqr
    size_t off_evpart;                                  // eval scratch
    size_t off_evdf;                                    // eval: double-float parameters and coefficients
    int64_t n_prm;                                      // feature parameters over all instances (doubles)
    int64_t n_fwd_items, n_col_items;                   // LSQR tile work items
    size_t off_fwd_items, off_col_items;
    size_t off_items, off_nitems, off_z, off_qblk;      // live column items, transposed-product scratch, block of each block row
    size_t off_tu;                                      // u~ on the block rows in operator precision
    size_t off_fitems, off_nfitems;                     // live forward items (128-row tiles)
    int64_t n_slots;                                    // column items per block at most (ceil(max_K / 8))
    int64_t n_t_items;                                  // fused product items: column chunks + 32-row tiles (bound)
    size_t off_titems, off_ntitems;
    size_t off_bcnt;                                    // per block: chunks of the transposed product finished (64-bit, monotone)
    size_t off_qord;                                    // QR launch order of the blocks (largest first)
    size_t off_yacc, off_rres, off_itn, off_scal0;      // refinement: accumulated y, FP64 residual, iterations,
                                                        // the first solve's scalars
    size_t total;
    int asm_prec, op;
};

// ---------------------------------------------------------------------------
// host-side helpers (plan.cu)
// ---------------------------------------------------------------------------
struct HostPlan {
    Layout L;
    InstRec *inst;       // n_inst
    BlkRec *blk;         // n_blocks
    int32_t *tile_blk;   // n_tiles: block of each 32-row tile
    int32_t *tile_row;   // n_tiles: first block-local row of the tile
    int32_t *cov;        // per-dimension cover tables: first covering subdomain, count (pairs)
    int32_t *fwd_items;  // (block, first row) of every 128-row tile
    int32_t *col_items;  // (block, first column) of every 8-column tile
    int32_t *qr_order;   // n_blocks: blocks by decreasing QR work (m K min(m, K)), ties by index
};

constexpr int kFwdRows = 128;  // rows of a forward (A x) work item (one warp)
// Columns per chunk of the transposed product (one warp per chunk).
__host__ __device__ inline int tchunk_cols(int ldm, int elem_bytes) {
    (void)ldm;
    (void)elem_bytes;
    return 8;
}
constexpr int kColTile = 8;    // columns of a transpose (A^T u) work item (one warp)

// Builds the plan (validates, computes records and layout).  Returns RFM_OK or
// RFM_EINVAL with the reason in err.
rfm_status build_plan(const rfm_problem *probs, int n_inst, const rfm_config *cfg, HostPlan *out, char *err,
                      size_t errlen);
void free_plan(HostPlan *p);
void host_block_rows(const HostPlan &P, int64_t b, int64_t *rows);

void set_error(const char *fmt, ...);

// Buffers of one batched QR-with-threshold pass (rrqr.cu): the system's own
// filter, or the fit of predicted values through the kept features.
struct FilterBufs {
    const BlkRec *blk;
    const int32_t *order;   // launch order of the blocks in the cluster kernels (null: natural)
    const void *M;          // input blocks (FP32 or FP64), ldm x K each
    double *W, *tau, *r11;  // QR work (R above the diagonal, reflectors below)
    int32_t *perm, *rank;
    double *Op;             // FP64 output arena (Q_hat, or the gathered kept columns)
    double *Q64;            // = Op when Q_hat is wanted in FP64
    float *Q32;             // Q_hat rounded to FP32
    bool gather;            // write the kept columns into Op instead of Q_hat
    bool fit;               // profiling label only
    bool no_cluster;        // test hook: the global-memory kernels only
    int64_t n_blocks, max_m, max_K;
};
rfm_status launch_filter_bufs(const FilterBufs &F, bool fp32, double tol, cudaStream_t st);
// The plan's QR launch order in the workspace, or null when RFM_OPT_QR_ORDER = 0.
const int32_t *qr_order_ptr(void *ws, const Layout &L);

template <typename T>
__host__ __device__ inline T *ws_ptr(void *ws, size_t off) {
    return reinterpret_cast<T *>(reinterpret_cast<char *>(ws) + off);
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------

// Grid coordinate lo + (g + 1/2) (hi - lo) / n, rounded step by step exactly as
// the host computes it (no contraction into FMA).
__host__ __device__ inline double grid_coord(double lo, double hi, int n, int64_t g) {
#ifdef __CUDA_ARCH__
    return __dadd_rn(lo, __ddiv_rn(__dmul_rn(__dadd_rn((double)g, 0.5), __dsub_rn(hi, lo)), (double)n));
#else
    volatile double a = (double)g + 0.5;
    volatile double b = a * (hi - lo);
    volatile double c = b / (double)n;
    return lo + c;
#endif
}

// Centre and half-width of subdomain ji along a dimension (Sec. 4.2).
__host__ __device__ inline void sub_geom(double lo, double hi, int S, double delta, int ji, double *mu, double *sig) {
#ifdef __CUDA_ARCH__
    double L = __dsub_rn(hi, lo);
    *mu = __dadd_rn(lo, __ddiv_rn(__dmul_rn(L, (double)ji), (double)(S - 1)));
    *sig = __ddiv_rn(__dmul_rn(L, delta), __dmul_rn(2.0, (double)(S - 1)));
#else
    volatile double L = hi - lo;
    volatile double a = L * (double)ji;
    volatile double b = a / (double)(S - 1);
    *mu = lo + b;
    volatile double c = L * delta;
    volatile double d = 2.0 * (double)(S - 1);
    *sig = c / d;
#endif
}

__device__ inline uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace rfm

#define RFM_CUDA_CHECK(call)                                                                        \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            rfm::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return RFM_ECUDA;                                                                       \
        }                                                                                           \
    } while (0)
