// lsqr_multi.cu -- LSQR (Paige and Saunders 1982) for many right-hand sides
// on one operator: the instances of a parametric family that share the
// decomposition and the features (only the data f, g differ) share M_hat,
// R_hat and Q_hat (Algorithm 1 and Proposition 3.1 depend on M alone), so
// the products of every right-hand side's iteration read the operator once:
//
//   forward     T_b = Q_hat_b V_b          (m_b x r_b) x (r_b x R) per block
//   transposed  Z_b = Q_hat_b^T U_b        (r_b x m_b) x (m_b x R) per block
//
// dense block products (CUDA-core register tiles of 64 x 64 outputs, 4 x 4 per
// thread, FP32 with FP32 accumulation for the FP32 Q_hat, FP64 for the FP64
// one).  Each right-hand side keeps its own LSQR scalars, estimates and
// stopping test; vectors are FP64, stored with the right-hand sides fastest
// ([row][R], [slot][R]).  One iteration is a fixed sequence of launches:
//   fwd -> rows (u~, ||u~||^2 partials) -> beta -> trans -> cols (v~,
//   ||v~||^2 partials) -> alpha (rotation, estimates, stopping) -> update
//   (y, w, ||y||^2 partials).
// Reductions are per-CTA partials summed in a fixed order: bitwise
// reproducible.
#include <string.h>

#include <vector>

#include "device.cuh"
#include "tc.cuh"
#include "prof.cuh"

namespace rfm {

rfm_status launch_coefficients(const HostPlan &P, void *ws, const double *y, double *a_out, cudaStream_t st,
                               int nsets = 1);

constexpr int kMT = 64;     // rows (forward) or columns (transposed) of a CTA tile
constexpr int kMR = 64;     // right-hand sides of a CTA tile
constexpr int kMK = 16;     // reduction depth of one shared-memory stage
constexpr int kMaxRhs = 256;
constexpr int kRedCtas = 512;   // CTAs of the row / column phases (partial sums)
constexpr int kMSets = 64, kMSub = 8;   // scalar kernels: sets per CTA, threads per set (m_sum)

struct MScal {
    double alpha, beta, rhobar, phibar, anorm2, bnorm, rnorm, arnorm, ynorm;
    double phi_rho, theta_rho, c, inv_alpha, inv_beta, inv_alpha_old, beta_old;
    double r0norm, hnorm, r0w;  // reported start residual; ||h||, ||h - Op y0|| of a given start
    int32_t itn, istop, done, start;   // start: 1 when the set keeps its warm start
};

struct MLayout {
    int R;
    int64_t n_fitems, n_titems;
    size_t off_inst, off_fitems, off_titems, off_vt, off_w, off_y, off_z, off_u, off_t, off_out, off_part, off_scal;
    size_t off_alive;
    size_t off_v32, off_u32;   // FP32 copies of v~ and u~ for the tensor-core products
    size_t total;
};

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

static MLayout multi_layout(const HostPlan &P, int R) {
    const Layout &L = P.L;
    MLayout M;
    memset(&M, 0, sizeof(M));
    M.R = R;
    int64_t nf = 0, nt = 0;
    for (int64_t b = 0; b < L.n_blocks; ++b) {
        nf += (P.blk[b].m + kMT - 1) / kMT;
        nt += (P.blk[b].K + kMT - 1) / kMT;
    }
    M.n_fitems = nf;
    M.n_titems = nt;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = al256(o + bytes); return r; };
    M.off_inst = take(sizeof(InstRec) * kMaxRhs);
    M.off_fitems = take(sizeof(int32_t) * 2 * (nf + 1));
    M.off_titems = take(sizeof(int32_t) * 2 * (nt + 1));
    const size_t cols = (size_t)L.n_cols * R * sizeof(double);
    M.off_vt = take(cols);
    M.off_w = take(cols);
    M.off_y = take(cols);
    M.off_z = take(cols);
    M.off_u = take((size_t)L.n_rows * R * sizeof(double));
    M.off_t = take((size_t)L.block_rows * R * sizeof(double));
    M.off_out = take(cols);
    M.off_part = take(sizeof(double) * 2 * kRedCtas * R);
    M.off_v32 = take((size_t)L.n_cols * R * sizeof(float));
    M.off_u32 = take((size_t)L.n_rows * R * sizeof(float));
    M.off_scal = take(sizeof(MScal) * R);
    M.off_alive = take(sizeof(int) * ((R + kMSets - 1) / kMSets));
    M.total = o;
    return M;
}

size_t multi_workspace_bytes(const HostPlan &P, int R) { return multi_layout(P, R).total; }

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// U[g][j] = H[j][g] (right-hand sides fastest), ||b_j||^2 partials
__global__ void __launch_bounds__(256) k_m_load(const double *__restrict__ H, int64_t n_rows, int R,
                                                double *__restrict__ U, double *__restrict__ part, float *__restrict__ U32) {
    __shared__ double red[256];
    const int Rp = R <= 1 ? 1 : (R <= 2 ? 2 : (R <= 4 ? 4 : (R <= 8 ? 8 : (R <= 16 ? 16 : (R <= 32 ? 32 : (R <= 64 ? 64 : (R <= 128 ? 128 : 256)))))));
    const int j = threadIdx.x % Rp, sub = threadIdx.x / Rp, nsub = 256 / Rp;
    double ss = 0.0;
    if (j < R)
        for (int64_t g = (int64_t)blockIdx.x * nsub + sub; g < n_rows; g += (int64_t)gridDim.x * nsub) {
            const double v = H[(int64_t)j * n_rows + g];
            U[g * R + j] = v;
            if (U32) U32[g * R + j] = (float)v;
            ss = fma(v, v, ss);
        }
    red[threadIdx.x] = ss;
    __syncthreads();
    if (threadIdx.x < Rp && j < R) {
        double t = 0.0;
        for (int s = 0; s < nsub; ++s) t += red[s * Rp + threadIdx.x];
        part[(int64_t)blockIdx.x * R + threadIdx.x] = t;
    }
}

// true once every right-hand side has stopped: k_m_beta writes one flag per
// CTA of 64 sets (nonzero while one of them still iterates); the heavy
// kernels then return at once (uniform over the CTA)
__device__ inline bool m_all_done(const int *__restrict__ alive, int ngs) {
    for (int g = 0; g < ngs; ++g)
        if (alive[g]) return false;
    return true;
}

// T = Q_hat_b (V / alpha) for one 64-row tile of one block and 64 right-hand
// sides (blockIdx.y); rows past the block and slots past its rank read 0.
template <typename TA>
__global__ void __launch_bounds__(256) k_m_fwd(const BlkRec *__restrict__ blks, const int32_t *__restrict__ items,
                                               const int32_t *__restrict__ rank, const TA *__restrict__ Q,
                                               const double *__restrict__ VT, const MScal *__restrict__ sc, int R,
                                               double *__restrict__ T,
                                               const int *__restrict__ alive, int ngs) {
    if (m_all_done(alive, ngs)) return;   // every right-hand side has stopped (uniform)
    __shared__ TA As[kMK][kMT], Bs[kMK][kMR];
    const int b = items[2 * blockIdx.x], r0 = items[2 * blockIdx.x + 1];
    const BlkRec &B = blks[b];
    const int rb = rank[b], m = B.m, j0 = blockIdx.y * kMR;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    TA acc[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] = (TA)0;
    for (int c0 = 0; c0 < rb; c0 += kMK) {
        for (int e = tid; e < kMK * kMT; e += 256) {
            const int col = e / kMT, row = e % kMT;
            As[col][row] = (c0 + col < rb && r0 + row < m) ? Q[B.moff + (int64_t)(c0 + col) * B.ldm + r0 + row] : (TA)0;
            const int jj = e % kMR, cc = e / kMR;
            Bs[cc][jj] = (c0 + cc < rb && j0 + jj < R)
                             ? (TA)(VT[(B.coff + c0 + cc) * R + j0 + jj] * sc[j0 + jj].inv_alpha)
                             : (TA)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kMK; ++kk) {
            TA a[4], v[4];
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
            for (int j = 0; j < 4; ++j) v[j] = Bs[kk][tx * 4 + j];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * v[j];
        }
        __syncthreads();
    }
    for (int i = 0; i < 4; ++i) {
        const int row = r0 + ty * 4 + i;
        if (row >= m) continue;
        for (int j = 0; j < 4; ++j) {
            const int jj = j0 + tx * 4 + j;
            if (jj < R) T[(B.roff + row) * R + jj] = (double)acc[i][j];
        }
    }
}

// Z = Q_hat_b^T (U_b / beta) for one 64-column tile of one block (columns
// below its rank) and 64 right-hand sides; U_b gathered by the block's rows.
template <typename TA>
__global__ void __launch_bounds__(256) k_m_trans(const BlkRec *__restrict__ blks, const int32_t *__restrict__ items,
                                                 const int32_t *__restrict__ rank, const int32_t *__restrict__ grow,
                                                 const TA *__restrict__ Q, const double *__restrict__ U,
                                                 const MScal *__restrict__ sc, int R, int64_t row_base,
                                                 double *__restrict__ Z,
                                                 const int *__restrict__ alive, int ngs) {
    if (m_all_done(alive, ngs)) return;   // every right-hand side has stopped (uniform)
    __shared__ TA As[kMK][kMT], Bs[kMK][kMR];
    __shared__ int64_t s_g[kMK];
    const int b = items[2 * blockIdx.x], c0 = items[2 * blockIdx.x + 1];
    const BlkRec &B = blks[b];
    const int rb = rank[b], m = B.m, j0 = blockIdx.y * kMR;
    if (c0 >= rb) return;   // uniform over the CTA
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    TA acc[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] = (TA)0;
    for (int i0 = 0; i0 < m; i0 += kMK) {
        if (tid < kMK) s_g[tid] = i0 + tid < m ? (int64_t)grow[B.roff + i0 + tid] - row_base : -1;
        __syncthreads();
        for (int e = tid; e < kMK * kMT; e += 256) {
            const int col = e / kMK, row = e % kMK;
            As[row][col] = (c0 + col < rb && i0 + row < m) ? Q[B.moff + (int64_t)(c0 + col) * B.ldm + i0 + row] : (TA)0;
            const int rr = e / kMR, jj = e % kMR;
            const int64_t g = s_g[rr];
            Bs[rr][jj] = (g >= 0 && j0 + jj < R) ? (TA)(U[g * R + j0 + jj] * sc[j0 + jj].inv_beta) : (TA)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kMK; ++kk) {
            TA a[4], v[4];
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
            for (int j = 0; j < 4; ++j) v[j] = Bs[kk][tx * 4 + j];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * v[j];
        }
        __syncthreads();
    }
    for (int i = 0; i < 4; ++i) {
        const int col = c0 + ty * 4 + i;
        if (col >= rb) continue;
        for (int j = 0; j < 4; ++j) {
            const int jj = j0 + tx * 4 + j;
            if (jj < R) Z[(B.coff + col) * R + jj] = (double)acc[i][j];
        }
    }
}

// ---------------------------------------------------------------------------
// Tensor-core block products of the FP32 operator (tcgen05, kind::f16): a CTA
// forms one 128 x 64 tile of T = Q_hat_b (V / alpha) (128 rows of a block, 64
// right-hand sides) or of Z = Q_hat_b^T (U_b / beta) (128 kept columns, 64
// right-hand sides) in tensor memory.  The FP32 operands are split into three
// BF16 terms as they are staged (bf16_split3) and the six products of terms
// whose orders add up to at most 2 are accumulated in FP32, which keeps the
// products at FP32 accuracy.  The vectors come from FP32 copies that the
// kernels producing v~ and u~ write (one conversion per element and
// iteration, not one per tile that reads it); 1 / alpha and 1 / beta scale
// the finished products.  Per 64-deep K chunk the 256 threads store A
// (128 x 64) and B (64 x 64) in the K-major layout from registers, one thread
// issues the 4 x 6 MMAs (K = 16 each) and commits them to an mbarrier, and
// while they run every thread loads its part of the next chunk into
// registers (48 loads in flight per thread: the loads' latency, not the
// MMAs, bounds the products); every thread then waits (bounded) and adds its
// part of the chunk's product (warps w and w + 4: TMEM lanes 32 (w mod 4) ..
// + 31, columns 32 (w / 4) .. + 31) to FP32 registers, so the tensor memory
// sums only 64 products at a time (its accumulation truncates: over whole
// blocks of thousands of rows it lost about a decade against the CUDA cores'
// FP32 sums).  The finished tile goes out through shared memory, one warp
// per output row of 64 consecutive doubles.  A wait that runs out gives NaN
// outputs.
// ---------------------------------------------------------------------------
constexpr int kTM = 128;                  // rows of D (block rows, or kept columns)
constexpr int kTN = 64;                   // right-hand sides per CTA
constexpr int kTK = 64;                   // K per staged chunk
constexpr int kTA = kTM * kTK * 2;        // bytes of one BF16 split of A
constexpr int kTB = kTN * kTK * 2;        // bytes of one BF16 split of B
constexpr int kTSmem = 3 * kTA + 3 * kTB; // dynamic shared memory

// every thread's staging of the chunk is in shared memory: one thread issues
// the 4 x 6 MMAs of the chunk and commits them to the mbarrier
__device__ inline void tcm_issue(unsigned char *sA, unsigned char *sB, uint32_t tmem, uint64_t *mbar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x == 0) {
        constexpr uint32_t idesc = tcm_idesc(kTM, kTN);
        const int sa[6] = {0, 0, 1, 0, 1, 2}, sb[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
        for (int kk = 0; kk < kTK / 16; ++kk)
#pragma unroll
            for (int t = 5; t >= 0; --t)   // smallest terms first
                tcm_mma(tmem, tcm_desc<kTK>(sA + sa[t] * kTA + kk * 256), tcm_desc<kTK>(sB + sb[t] * kTB + kk * 256),
                        idesc, (kk > 0 || t < 5) ? 1u : 0u);
        tcm_commit(mbar);
    }
}

// bounded wait for the chunk's MMAs (ok = false when it runs out); the
// operands in shared memory are free afterwards
__device__ inline void tcm_finish(uint64_t *mbar, unsigned &parity, bool &ok) {
    const bool got = __syncthreads_and(tcm_wait(mbar, parity));
    if (!got) {
        (void)tcm_wait(mbar, parity);   // MMAs still in flight: a second bounded wait
        ok = false;
    }
    parity ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// acc += this thread's 32 columns of the chunk's product (TMEM lanes 32 (w mod
// 4) .. + 31 for warps w and w + 4, columns 32 (w / 4) .. + 31), 16 at a time
__device__ inline void tcm_accumulate(uint32_t tmem, float (&acc)[32]) {
    const int warp = threadIdx.x >> 5;
    const uint32_t a = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * (warp >> 2));
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float v[16];
        tcm_ld16(a + 16 * h, v);
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[16 * h + q] += v[q];
    }
}

// The finished 128 x 64 tile leaves through shared memory (the operand
// buffers, free once the last MMAs completed), rows padded to 65 doubles, so
// that each output row's 64 consecutive doubles are written by one warp.
constexpr int kTLd = kTN + 1;
static_assert(kTM * kTLd * 8 <= kTSmem, "output tile fits the operand buffers");

__device__ inline void tcm_tile_to_smem(double *stile, const float (&acc)[32], const MScal *__restrict__ sc,
                                        bool by_alpha, int j0, int R, bool ok) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lr = 32 * (warp & 3) + lane, lc = 32 * (warp >> 2);
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        const int j = j0 + lc + q;
        const double s = j < R ? (by_alpha ? sc[j].inv_alpha : sc[j].inv_beta) : 0.0;
        stile[lr * kTLd + lc + q] = ok ? (double)acc[q] * s : __longlong_as_double(0x7ff8000000000000ll);
    }
    __syncthreads();
}

__device__ inline uint32_t tcm_setup(uint64_t *mbar, uint32_t *tmem_slot) {
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tcm_su32(tmem_slot)),
                     "r"(kTN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tcm_su32(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return *tmem_slot;
}

__device__ inline void tcm_teardown(uint32_t tmem) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTN) : "memory");
}

// T = Q_hat_b (V / alpha) for 128 rows of one block (items: block, first row).
// Each thread stages 4 core-matrix rows of A (row tid mod 128, column groups
// tid / 128 + 2i) and 2 of B (data set tid mod 64, column groups tid / 64 +
// 4i); the next chunk's 48 loads are issued while the current chunk's MMAs
// run.
__global__ void __launch_bounds__(256, 2) k_m_fwd_tc(const BlkRec *__restrict__ blks, const int32_t *__restrict__ items,
                                                     const int32_t *__restrict__ rank, const float *__restrict__ Q,
                                                     const float *__restrict__ V32, const MScal *__restrict__ sc, int R,
                                                     double *__restrict__ T,
                                                     const int *__restrict__ alive, int ngs) {
    if (m_all_done(alive, ngs)) return;   // every right-hand side has stopped (uniform)
    extern __shared__ __align__(128) unsigned char tsm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    unsigned char *sA = tsm, *sB = tsm + 3 * kTA;
    const int b = items[2 * blockIdx.x], r0 = items[2 * blockIdx.x + 1];
    const BlkRec &B = blks[b];
    const int rb = rank[b], m = B.m, ldm = B.ldm, j0 = blockIdx.y * kTN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (rb <= 0) {   // no kept columns: the rows' partials are zero (uniform over the CTA)
        const int row = r0 + 32 * (warp & 3) + lane, jc = j0 + 32 * (warp >> 2);
        if (row < m)
            for (int q = 0; q < 32; ++q)
                if (jc + q < R) T[(B.roff + row) * R + jc + q] = 0.0;
        return;
    }
    const uint32_t tmem = tcm_setup(&mbar, &tmem_slot);
    unsigned parity = 0;
    bool ok = true;
    float acc[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) acc[q] = 0.f;
    const int ra = tid & (kTM - 1), ga = tid >> 7;    // A: row, first column group
    const int nb = tid & (kTN - 1), gb = tid >> 6;    // B: data set, first column group
    const bool row_in = r0 + ra < m, set_in = j0 + nb < R;
    const float *qa = Q + B.moff + r0 + ra;
    const float *vb = V32 + (int64_t)B.coff * R + j0 + nb;
    float xa[4][8], xb[2][8];
    auto load = [&](int c0) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = c0 + 8 * (ga + 2 * i) + q;
                xa[i][q] = (k < rb && row_in) ? __ldg(qa + (int64_t)k * ldm) : 0.f;
            }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = c0 + 8 * (gb + 4 * i) + q;
                xb[i][q] = (k < rb && set_in) ? vb[(int64_t)k * R] : 0.f;   // v~ (scaled by 1 / alpha below)
            }
    };
    load(0);
    for (int c0 = 0; c0 < rb && ok; c0 += kTK) {
#pragma unroll
        for (int i = 0; i < 4; ++i) tcm_store8(sA, tcm_off<kTK>(ra, 8 * (ga + 2 * i)), kTA, xa[i]);
#pragma unroll
        for (int i = 0; i < 2; ++i) tcm_store8(sB, tcm_off<kTK>(nb, 8 * (gb + 4 * i)), kTB, xb[i]);
        tcm_issue(sA, sB, tmem, &mbar);
        if (c0 + kTK < rb) load(c0 + kTK);
        tcm_finish(&mbar, parity, ok);
        tcm_accumulate(tmem, acc);
    }
    double *stile = reinterpret_cast<double *>(tsm);
    tcm_tile_to_smem(stile, acc, sc, true, j0, R, ok);
    const int nj = min(kTN, R - j0);
    for (int lr = warp; lr < kTM && r0 + lr < m; lr += 8)
        for (int jj = lane; jj < nj; jj += 32) T[(B.roff + r0 + lr) * R + j0 + jj] = stile[lr * kTLd + jj];
    tcm_teardown(tmem);
}

// Z = Q_hat_b^T (U_b / beta) for 128 kept columns of one block (items: block,
// first column); U_b gathered by the block's rows.  Staging as in k_m_fwd_tc:
// 4 core-matrix rows of A (kept column tid mod 128, row groups tid / 128 +
// 2i, two 16-byte loads each) and 2 of B (data set tid mod 64, row groups
// tid / 64 + 4i), the next chunk's loads issued while the MMAs run.
__global__ void __launch_bounds__(256, 2) k_m_trans_tc(const BlkRec *__restrict__ blks, const int32_t *__restrict__ items,
                                                       const int32_t *__restrict__ rank, const int32_t *__restrict__ grow,
                                                       const float *__restrict__ Q, const float *__restrict__ U32,
                                                       const MScal *__restrict__ sc, int R, double *__restrict__ Z,
                                                       const int *__restrict__ alive, int ngs) {
    if (m_all_done(alive, ngs)) return;   // every right-hand side has stopped (uniform)
    extern __shared__ __align__(128) unsigned char tsm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    unsigned char *sA = tsm, *sB = tsm + 3 * kTA;
    const int b = items[2 * blockIdx.x], c0 = items[2 * blockIdx.x + 1];
    const BlkRec &B = blks[b];
    const int rb = rank[b], m = B.m, ldm = B.ldm, j0 = blockIdx.y * kTN;
    if (c0 >= rb || m <= 0) return;   // uniform over the CTA
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t tmem = tcm_setup(&mbar, &tmem_slot);
    unsigned parity = 0;
    bool ok = true;
    float acc[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) acc[q] = 0.f;
    const int ca = tid & (kTM - 1), ga = tid >> 7;    // A: kept column, first row group
    const int nb = tid & (kTN - 1), gb = tid >> 6;    // B: data set, first row group
    const bool col_in = c0 + ca < rb, set_in = j0 + nb < R;
    const float *qa = Q + B.moff + (int64_t)(c0 + ca) * ldm;
    const int32_t *gr = grow + B.roff;
    const float *ub = U32 + j0 + nb;
    float xa[4][8], xb[2][8];
    auto load = [&](int i0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = i0 + 8 * (ga + 2 * i);
            if (col_in && r < ldm) {   // ldm is a multiple of 32: the 8 rows lie inside the column
                const float4 *src = reinterpret_cast<const float4 *>(qa + r);
                const float4 p = __ldg(src), q4 = __ldg(src + 1);
                xa[i][0] = p.x; xa[i][1] = p.y; xa[i][2] = p.z; xa[i][3] = p.w;
                xa[i][4] = q4.x; xa[i][5] = q4.y; xa[i][6] = q4.z; xa[i][7] = q4.w;
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (r + q >= m) xa[i][q] = 0.f;
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) xa[i][q] = 0.f;
            }
        }
        int g[2][8];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int r = i0 + 8 * (gb + 4 * i) + q;
                g[i][q] = (r < m && set_in) ? __ldg(gr + r) : -1;
            }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int q = 0; q < 8; ++q)
                xb[i][q] = g[i][q] >= 0 ? ub[(int64_t)g[i][q] * R] : 0.f;   // u~ (scaled by 1 / beta below)
    };
    load(0);
    for (int i0 = 0; i0 < m && ok; i0 += kTK) {
#pragma unroll
        for (int i = 0; i < 4; ++i) tcm_store8(sA, tcm_off<kTK>(ca, 8 * (ga + 2 * i)), kTA, xa[i]);
#pragma unroll
        for (int i = 0; i < 2; ++i) tcm_store8(sB, tcm_off<kTK>(nb, 8 * (gb + 4 * i)), kTB, xb[i]);
        tcm_issue(sA, sB, tmem, &mbar);
        if (i0 + kTK < m) load(i0 + kTK);
        tcm_finish(&mbar, parity, ok);
        tcm_accumulate(tmem, acc);
    }
    double *stile = reinterpret_cast<double *>(tsm);
    tcm_tile_to_smem(stile, acc, sc, false, j0, R, ok);
    const int nj = min(kTN, R - j0);
    for (int lc = warp; lc < kTM && c0 + lc < rb; lc += 8)
        for (int jj = lane; jj < nj; jj += 32) Z[(B.coff + c0 + lc) * R + j0 + jj] = stile[lc * kTLd + jj];
    tcm_teardown(tmem);
}

__device__ inline int pow2_at_least(int R) {
    int p = 1;
    while (p < R) p <<= 1;
    return p;
}

// per-CTA partial sums of one value per right-hand side (threads (sub, j))
__device__ inline void m_partials(double v, int R, double *red, double *part) {
    const int Rp = pow2_at_least(R), nsub = 256 / Rp;
    red[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x < R) {
        double t = 0.0;
        for (int s = 0; s < nsub; ++s) t += red[s * Rp + threadIdx.x];
        part[(int64_t)blockIdx.x * R + threadIdx.x] = t;
    }
}

// The scalar kernels run kMSub threads per right-hand side (kMSets sets per
// CTA): thread sub of set j sums the partials of CTAs sub, sub + kMSub, ...,
// and the kMSub sums are combined in sub order, so the result is fixed for a
// given partial count; valid in the sub = 0 threads.  Every thread of the CTA
// calls it (it synchronises).
__device__ inline double m_sum(const double *part, int nctas, int R, int j, double (*red)[kMSets]) {
    const int js = threadIdx.x % kMSets, sub = threadIdx.x / kMSets;
    double t = 0.0;
    if (j < R)
        for (int c = sub; c < nctas; c += kMSub) t += part[(int64_t)c * R + j];
    red[sub][js] = t;
    __syncthreads();
    double s = 0.0;
    if (sub == 0)
        for (int u = 0; u < kMSub; ++u) s += red[u][js];
    __syncthreads();
    return s;
}

// Warm starts.  VT and Y = Y0 (sets contiguous in Y0) on the kept slots, 0
// elsewhere; inv_alpha = 1 so that the forward kernel forms T = Op Y0.
__global__ void __launch_bounds__(256) k_m_in(const double *__restrict__ Y0, const int32_t *__restrict__ rank,
                                              int64_t n_cols, int K, int R, double *__restrict__ VT,
                                              double *__restrict__ Y, MScal *__restrict__ sc, float *__restrict__ V32) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_cols * R;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t slot = e / R;
        const int j = (int)(e % R);
        const double v = (int)(slot % K) < rank[slot / K] ? Y0[(int64_t)j * n_cols + slot] : 0.0;
        VT[e] = v;
        if (V32) V32[e] = (float)v;
        Y[e] = v;
    }
    if (blockIdx.x == 0)
        for (int j = threadIdx.x; j < R; j += blockDim.x) sc[j].inv_alpha = 1.0;
}

// u = h - (sum over the row's block rows of T); partials of ||u||^2 (part)
// and of ||h||^2 (part + gridDim.x R)
__global__ void __launch_bounds__(256) k_m_load_warm(const InstRec *__restrict__ insts,
                                                     const int32_t *__restrict__ rowlist, const double *__restrict__ H,
                                                     const double *__restrict__ T, int R, double *__restrict__ U,
                                                     double *__restrict__ part, float *__restrict__ U32) {
    __shared__ double red[256];
    const InstRec &I = insts[0];
    const int Rp = pow2_at_least(R), j = threadIdx.x % Rp, sub = threadIdx.x / Rp, nsub = 256 / Rp;
    double su = 0.0, sh = 0.0;
    if (j < R)
        for (int64_t g = (int64_t)blockIdx.x * nsub + sub; g < I.N; g += (int64_t)gridDim.x * nsub) {
            const int32_t *lst = rowlist + I.rl_off + g * I.C;
            double s = 0.0;
            for (int e = 0; e < I.C; ++e) {
                const int q = lst[e];
                if (q >= 0) s += T[(int64_t)q * R + j];
            }
            const double h = H[(int64_t)j * I.N + g], u = h - s;
            U[g * R + j] = u;
            if (U32) U32[g * R + j] = (float)u;
            su = fma(u, u, su);
            sh = fma(h, h, sh);
        }
    m_partials(su, R, red, part);
    __syncthreads();
    m_partials(sh, R, red, part + (int64_t)gridDim.x * R);
}

// per set: keep the warm start when ||h - Op y0|| < ||h||, else fall back to
// the zero start (the rule of rfm_lsqr_solve)
__global__ void __launch_bounds__(kMSets * kMSub) k_m_start(MScal *__restrict__ sc, const double *__restrict__ part,
                                                             int nctas, int R) {
    __shared__ double red[kMSub][kMSets];
    const int j = blockIdx.x * kMSets + threadIdx.x % kMSets;
    const double r2 = m_sum(part, nctas, R, j, red), h2 = m_sum(part + (int64_t)nctas * R, nctas, R, j, red);
    if (threadIdx.x >= kMSets || j >= R) return;
    const double r0 = sqrt(r2), hn = sqrt(h2);
    sc[j].r0w = r0;
    sc[j].hnorm = hn;
    sc[j].start = r0 < hn ? 1 : 0;
}

// the sets that fall back: u = h, y = 0
__global__ void __launch_bounds__(256) k_m_fallback(const MScal *__restrict__ sc, const double *__restrict__ H,
                                                    int64_t n_rows, int64_t n_cols, int R, double *__restrict__ U,
                                                    double *__restrict__ Y, float *__restrict__ U32) {
    const int64_t nr = n_rows * R, nt = nr + n_cols * R;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nt; e += (int64_t)gridDim.x * blockDim.x) {
        if (e < nr) {
            const int64_t g = e / R;
            const int j = (int)(e % R);
            if (!sc[j].start) {
                U[e] = H[(int64_t)j * n_rows + g];
                if (U32) U32[e] = (float)U[e];
            }
        } else {
            const int j = (int)((e - nr) % R);
            if (!sc[j].start) Y[e - nr] = 0.0;
        }
    }
}

// partials of ||u||^2 (after the fallback)
__global__ void __launch_bounds__(256) k_m_unorm(const double *__restrict__ U, int64_t n_rows, int R,
                                                 double *__restrict__ part) {
    __shared__ double red[256];
    const int Rp = pow2_at_least(R), j = threadIdx.x % Rp, sub = threadIdx.x / Rp, nsub = 256 / Rp;
    double ss = 0.0;
    if (j < R)
        for (int64_t g = (int64_t)blockIdx.x * nsub + sub; g < n_rows; g += (int64_t)gridDim.x * nsub)
            ss = fma(U[g * R + j], U[g * R + j], ss);
    m_partials(ss, R, red, part);
}

// after the first beta: the stopping test's ||b|| is ||h||, and the given
// start's residual is reported (also when it was not kept, as rfm_lsqr_solve)
__global__ void k_m_fixb(MScal *__restrict__ sc, int R) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= R) return;
    sc[j].bnorm = sc[j].hnorm;
    sc[j].r0norm = sc[j].r0w;
}

// rows: u~ = sum over the row's block rows of T - alpha (u~ / beta), ||u~||^2
__global__ void __launch_bounds__(256) k_m_rows(const InstRec *__restrict__ insts, const int32_t *__restrict__ rowlist,
                                                const double *__restrict__ T, double *__restrict__ U,
                                                const MScal *__restrict__ sc, int R, double *__restrict__ part,
                                                float *__restrict__ U32,
                                                const int *__restrict__ alive, int ngs) {
    if (m_all_done(alive, ngs)) return;   // every right-hand side has stopped (uniform)
    __shared__ double red[256];
    const InstRec &I = insts[0];
    const int Rp = pow2_at_least(R), j = threadIdx.x % Rp, sub = threadIdx.x / Rp, nsub = 256 / Rp;
    double ss = 0.0;
    if (j < R) {
        const double al = sc[j].alpha, ib = sc[j].inv_beta;
        for (int64_t g = (int64_t)blockIdx.x * nsub + sub; g < I.N; g += (int64_t)gridDim.x * nsub) {
            const int32_t *lst = rowlist + I.rl_off + g * I.C;
            double s = 0.0;
            for (int e = 0; e < I.C; ++e) {
                const int q = lst[e];
                if (q >= 0) s += T[(int64_t)q * R + j];
            }
            const double u = s - al * (U[g * R + j] * ib);
            U[g * R + j] = u;
            if (U32) U32[g * R + j] = (float)u;
            ss = fma(u, u, ss);
        }
    }
    m_partials(ss, R, red, part);
}

// columns: v~ = Z (first pass) or Z - beta (v~_old / alpha_old), ||v~||^2
__global__ void __launch_bounds__(256) k_m_cols(const int32_t *__restrict__ rank,
                                                int64_t n_cols, int K, const double *__restrict__ Z,
                                                double *__restrict__ VT, const MScal *__restrict__ sc, int R,
                                                int first, double *__restrict__ part, float *__restrict__ V32,
                                                const int *__restrict__ alive, int ngs) {
    if (m_all_done(alive, ngs)) return;   // every right-hand side has stopped (uniform)
    __shared__ double red[256];
    const int Rp = pow2_at_least(R), j = threadIdx.x % Rp, sub = threadIdx.x / Rp, nsub = 256 / Rp;
    double ss = 0.0;
    if (j < R) {
        const double be = sc[j].beta, ia = sc[j].inv_alpha;
        for (int64_t s = (int64_t)blockIdx.x * nsub + sub; s < n_cols; s += (int64_t)gridDim.x * nsub) {
            if ((int)(s % K) >= rank[s / K]) continue;
            const double z = Z[s * R + j];
            const double v = first ? z : z - be * (VT[s * R + j] * ia);
            VT[s * R + j] = v;
            if (V32) V32[s * R + j] = (float)v;
            ss = fma(v, v, ss);
        }
    }
    m_partials(ss, R, red, part);
}

// the first nctas partial rows of part, summed in CTA order, per right-hand side

// The stopping test of the previous iteration k (its estimates, ||y_k|| from
// its update's partials; the tests of rfm_lsqr_solve), then beta = ||u~||.
__global__ void __launch_bounds__(kMSets * kMSub) k_m_beta(MScal *__restrict__ sc, const double *__restrict__ part,
                                                            int nctas, const double *__restrict__ ypart, int ynctas,
                                                            int R, int first, double atol, double btol,
                                                            int *__restrict__ alive) {
    __shared__ double red[kMSub][kMSets];
    const int j = blockIdx.x * kMSets + threadIdx.x % kMSets;
    const double b2 = m_sum(part, nctas, R, j, red);
    const double y2 = ypart ? m_sum(ypart, ynctas, R, j, red) : 0.0;
    auto set = [&]() {
        MScal &q = sc[j];
        if (!first && ypart) q.ynorm = sqrt(y2);
        if (q.done == 2) q.done = 1;
        if (!first && !q.done && q.itn > 0) {
            const double anorm = sqrt(q.anorm2);
            if (q.rnorm <= btol * q.bnorm + atol * anorm * q.ynorm) {
                q.done = 1;
                q.istop = 1;
            } else if (q.arnorm <= atol * anorm * q.rnorm) {
                q.done = 1;
                q.istop = 2;
            }
        }
        if (q.done) return;
        q.beta_old = q.beta;
        q.beta = sqrt(b2);
        q.inv_beta = q.beta > 0.0 ? 1.0 / q.beta : 0.0;
        if (first) {
            q.bnorm = q.beta;
            q.r0norm = q.beta;
            q.phibar = q.beta;
            q.rnorm = q.beta;
            q.istop = 7;
            q.itn = 0;
            q.done = 0;
        }
    };
    const bool mine = threadIdx.x < kMSets && j < R;
    if (mine) set();
    // a set that has stopped (done = 1) never iterates again: once no set of
    // the CTA is live, the flag stays 0 for the rest of the call
    const int live = __syncthreads_or(mine && sc[j].done == 0);
    if (threadIdx.x == 0) alive[blockIdx.x] = live;
}

// alpha = ||v~||, then the plane rotation of the iteration and the estimates
// of the 1982 paper (||B_k||_F^2 gains alpha_k^2 + beta_{k+1}^2); an exact
// stop (alpha or beta zero) or a non-finite scalar ends the right-hand side
// after this iteration's update (done = 2)
__global__ void __launch_bounds__(kMSets * kMSub) k_m_alpha(MScal *__restrict__ sc, const double *__restrict__ part,
                                                             int nctas, int R, int first, double atol, double btol,
                                                             int max_iter) {
    __shared__ double red[kMSub][kMSets];
    const int j = blockIdx.x * kMSets + threadIdx.x % kMSets;
    const double a2 = m_sum(part, nctas, R, j, red);
    if (threadIdx.x >= kMSets || j >= R) return;
    MScal &q = sc[j];
    if (!first && q.done) return;
    const double al = sqrt(a2);
    const double al_old = q.alpha;
    q.inv_alpha_old = q.inv_alpha;
    q.alpha = al;
    q.inv_alpha = al > 0.0 ? 1.0 / al : 0.0;
    if (first) {
        q.rhobar = al;
        q.arnorm = al * q.beta;
        q.anorm2 = 0.0;
        if (q.beta == 0.0 || al == 0.0) {
            q.done = 1;
            q.istop = 0;
        }
        return;
    }
    q.anorm2 += al_old * al_old + q.beta * q.beta;
    const double rho = sqrt(q.rhobar * q.rhobar + q.beta * q.beta);
    const double ir = 1.0 / rho;
    const double c = q.rhobar * ir, s = q.beta * ir;
    const double theta = s * al;
    q.rhobar = -c * al;
    const double phi = c * q.phibar;
    q.phibar = s * q.phibar;
    q.phi_rho = phi * ir;
    q.theta_rho = theta * ir;
    q.c = c;
    q.rnorm = q.phibar;
    q.arnorm = q.phibar * al * fabs(c);
    q.itn += 1;
    const double anorm = sqrt(q.anorm2);
    if (!isfinite(rho) || !isfinite(q.phibar)) {
        q.done = 2;
        q.istop = -1;
    } else if (al == 0.0 || q.beta == 0.0) {
        q.done = 2;
        q.istop = 0;
    }
    (void)anorm;
    (void)atol;
    (void)btol;
    (void)max_iter;
}

// v = v~ / alpha; first pass: w = v; then y += (phi/rho) w, w = v - (theta/rho) w; ||y||^2
__global__ void __launch_bounds__(256) k_m_update(const int32_t *__restrict__ rank, int64_t n_cols, int K,
                                                  const double *__restrict__ VT, double *__restrict__ W,
                                                  double *__restrict__ Y, const MScal *__restrict__ sc, int R,
                                                  int first, double *__restrict__ part,
                                                  const int *__restrict__ alive, int ngs) {
    if (m_all_done(alive, ngs)) return;   // every right-hand side has stopped (uniform)
    __shared__ double red[256];
    const int Rp = pow2_at_least(R), j = threadIdx.x % Rp, sub = threadIdx.x / Rp, nsub = 256 / Rp;
    double ss = 0.0;
    if (j < R) {
        const MScal &q = sc[j];
        const bool live = first || q.done != 1;
        for (int64_t s = (int64_t)blockIdx.x * nsub + sub; s < n_cols; s += (int64_t)gridDim.x * nsub) {
            if ((int)(s % K) >= rank[s / K]) continue;
            const int64_t o = s * R + j;
            double yv = Y[o];
            if (live) {
                const double v = VT[o] * q.inv_alpha;
                if (first) {
                    W[o] = v;
                } else {
                    const double wo = W[o];
                    yv = fma(q.phi_rho, wo, yv);
                    Y[o] = yv;
                    W[o] = fma(-q.theta_rho, wo, v);
                }
            }
            ss = fma(yv, yv, ss);
        }
    }
    m_partials(ss, R, red, part);
}

// out[j][s] = Y[s][j] (right-hand sides contiguous), and the reports
__global__ void k_m_out(const double *__restrict__ Y, int64_t n_cols, int R, double *__restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_cols * R; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = e / R;
        const int j = (int)(e % R);
        out[(int64_t)j * n_cols + s] = Y[e];
    }
}

__global__ void k_m_report(const MScal *__restrict__ sc, int R, rfm_lsqr_report *__restrict__ rep) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= R) return;
    const MScal &q = sc[j];
    rep[j].itn = q.itn;
    rep[j].istop = q.istop;
    rep[j].rnorm = q.rnorm;
    rep[j].arnorm = q.arnorm;
    rep[j].anorm = sqrt(q.anorm2);
    rep[j].ynorm = q.ynorm;
    rep[j].bnorm = q.bnorm;
    rep[j].status = q.istop < 0 ? (double)RFM_ENUMERIC : 0.0;
    rep[j].start = (double)q.start;
    rep[j].r0norm = q.r0norm;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static unsigned red_grid(int64_t n, int R) {
    int Rp = 1;
    while (Rp < R) Rp <<= 1;
    const int64_t per = 256 / Rp;
    int64_t g = (n + per - 1) / per;
    return (unsigned)(g < 1 ? 1 : (g > kRedCtas ? kRedCtas : g));
}

static int g_multi_tc = 1;   // FP32 operator: block products on the tensor cores (1) or the CUDA cores (0)
void set_multi_tc(int v) { g_multi_tc = v; }

rfm_status launch_lsqr_multi(const HostPlan &P, void *ws, const rfm_lsqr_opts *opts, int R, const double *H,
                             const double *Y0, double *A, rfm_lsqr_report *rep, void *mws, cudaStream_t st) {
    const Layout &L = P.L;
    if (L.n_inst != 1 || (L.op != RFM_OP_Q32 && L.op != RFM_OP_Q64)) {
        set_error("rfm_lsqr_multi: one instance with an explicit Q_hat operator (RFM_OP_Q32 or RFM_OP_Q64)");
        return RFM_EINVAL;
    }
    if (R < 1 || R > kMaxRhs) {
        set_error("rfm_lsqr_multi: 1..%d right-hand sides", kMaxRhs);
        return RFM_EINVAL;
    }
    const MLayout M = multi_layout(P, R);
    // the FP32 operator's products on the tensor cores (128-row / 128-column
    // tiles), the FP64 one's on the CUDA cores (64)
    const bool tc = L.op == RFM_OP_Q32 && g_multi_tc;
    const int tile = tc ? kTM : kMT;
    // work lists: (block, first row) of every row tile, (block, first column) of every column tile
    std::vector<int32_t> fi, ti;
    for (int64_t b = 0; b < L.n_blocks; ++b) {
        for (int r = 0; r < P.blk[b].m; r += tile) { fi.push_back((int32_t)b); fi.push_back(r); }
        for (int c = 0; c < P.blk[b].K; c += tile) { ti.push_back((int32_t)b); ti.push_back(c); }
    }
    int32_t *d_fi = ws_ptr<int32_t>(mws, M.off_fitems), *d_ti = ws_ptr<int32_t>(mws, M.off_titems);
    if (!fi.empty())
        RFM_CUDA_CHECK(cudaMemcpyAsync(d_fi, fi.data(), sizeof(int32_t) * fi.size(), cudaMemcpyHostToDevice, st));
    if (!ti.empty())
        RFM_CUDA_CHECK(cudaMemcpyAsync(d_ti, ti.data(), sizeof(int32_t) * ti.size(), cudaMemcpyHostToDevice, st));
    // (copies from pageable host memory are staged before cudaMemcpyAsync returns)
    double *VT = ws_ptr<double>(mws, M.off_vt), *W = ws_ptr<double>(mws, M.off_w), *Y = ws_ptr<double>(mws, M.off_y);
    double *Z = ws_ptr<double>(mws, M.off_z), *U = ws_ptr<double>(mws, M.off_u), *T = ws_ptr<double>(mws, M.off_t);
    double *part = ws_ptr<double>(mws, M.off_part), *ypart = part + (size_t)kRedCtas * R;
    MScal *sc = ws_ptr<MScal>(mws, M.off_scal);
    int *alive = ws_ptr<int>(mws, M.off_alive);
    float *V32 = tc ? ws_ptr<float>(mws, M.off_v32) : nullptr, *U32 = tc ? ws_ptr<float>(mws, M.off_u32) : nullptr;
    const size_t cols = (size_t)L.n_cols * R * sizeof(double);
    RFM_CUDA_CHECK(cudaMemsetAsync(sc, 0, sizeof(MScal) * R, st));
    RFM_CUDA_CHECK(cudaMemsetAsync(alive, 1, sizeof(int) * ((R + kMSets - 1) / kMSets), st));   // nonzero: every set live
    RFM_CUDA_CHECK(cudaMemsetAsync(Y, 0, cols, st));
    RFM_CUDA_CHECK(cudaMemsetAsync(VT, 0, cols, st));
    RFM_CUDA_CHECK(cudaMemsetAsync(W, 0, cols, st));
    const BlkRec *blks = ws_ptr<BlkRec>(ws, L.off_blk);
    const int32_t *rank = ws_ptr<int32_t>(ws, L.off_rank), *grow = ws_ptr<int32_t>(ws, L.off_grow);
    const InstRec *insts = ws_ptr<InstRec>(ws, L.off_inst);
    const int32_t *rowlist = ws_ptr<int32_t>(ws, L.off_rowlist);
    const int K = (int)P.inst[0].K;
    const unsigned gr = red_grid(L.n_rows, R), gc = red_grid(L.n_cols, R), gs = (unsigned)((R + kMSets - 1) / kMSets);
    const dim3 gf((unsigned)(fi.size() / 2), (unsigned)((R + kMR - 1) / kMR)),
        gt((unsigned)(ti.size() / 2), (unsigned)((R + kMR - 1) / kMR));
    if (tc) {
        RFM_CUDA_CHECK(cudaFuncSetAttribute(k_m_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTSmem));
        RFM_CUDA_CHECK(cudaFuncSetAttribute(k_m_trans_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTSmem));
    }
    const bool q32 = L.op == RFM_OP_Q32;
    const void *Q = q32 ? (const void *)ws_ptr<float>(ws, L.off_q32) : (const void *)ws_ptr<double>(ws, L.off_op);

    auto fwd = [&]() -> rfm_status {
        ProfScope ps("k_m_fwd", st);
        if (tc)
            k_m_fwd_tc<<<gf, 256, kTSmem, st>>>(blks, d_fi, rank, (const float *)Q, V32, sc, R, T, alive, (int)gs);
        else if (q32)
            k_m_fwd<float><<<gf, 256, 0, st>>>(blks, d_fi, rank, (const float *)Q, VT, sc, R, T, alive, (int)gs);
        else
            k_m_fwd<double><<<gf, 256, 0, st>>>(blks, d_fi, rank, (const double *)Q, VT, sc, R, T, alive, (int)gs);
        RFM_CUDA_CHECK(cudaGetLastError());
        return RFM_OK;
    };
    auto trans = [&]() -> rfm_status {
        ProfScope ps("k_m_trans", st);
        if (tc)
            k_m_trans_tc<<<gt, 256, kTSmem, st>>>(blks, d_ti, rank, grow, (const float *)Q, U32, sc, R, Z, alive, (int)gs);
        else if (q32)
            k_m_trans<float><<<gt, 256, 0, st>>>(blks, d_ti, rank, grow, (const float *)Q, U, sc, R, 0, Z, alive, (int)gs);
        else
            k_m_trans<double><<<gt, 256, 0, st>>>(blks, d_ti, rank, grow, (const double *)Q, U, sc, R, 0, Z, alive, (int)gs);
        RFM_CUDA_CHECK(cudaGetLastError());
        return RFM_OK;
    };
    rfm_status rc;
    // initialisation: beta_1 u_1 = h (or h - Op y0 for a kept warm start),
    // alpha_1 v_1 = A^T u_1, w_1 = v_1
    if (Y0) {
        ProfScope ps("k_m_warm", st);
        k_m_in<<<2048, 256, 0, st>>>(Y0, rank, L.n_cols, K, R, VT, Y, sc, V32);
        RFM_CUDA_CHECK(cudaGetLastError());
        if ((rc = fwd()) != RFM_OK) return rc;
        k_m_load_warm<<<gr, 256, 0, st>>>(insts, rowlist, H, T, R, U, part, U32);
        k_m_start<<<gs, kMSets * kMSub, 0, st>>>(sc, part, (int)gr, R);
        k_m_fallback<<<2048, 256, 0, st>>>(sc, H, L.n_rows, L.n_cols, R, U, Y, U32);
        k_m_unorm<<<gr, 256, 0, st>>>(U, L.n_rows, R, part);
        RFM_CUDA_CHECK(cudaGetLastError());
    } else {
        ProfScope ps("k_m_load", st);
        k_m_load<<<gr, 256, 0, st>>>(H, L.n_rows, R, U, part, U32);
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    k_m_beta<<<gs, kMSets * kMSub, 0, st>>>(sc, part, (int)gr, nullptr, 0, R, 1, opts->atol, opts->btol, alive);
    if (Y0) k_m_fixb<<<gs, 64, 0, st>>>(sc, R);
    if ((rc = trans()) != RFM_OK) return rc;
    k_m_cols<<<gc, 256, 0, st>>>(rank, L.n_cols, K, Z, VT, sc, R, 1, part, V32, alive, (int)gs);
    k_m_alpha<<<gs, kMSets * kMSub, 0, st>>>(sc, part, (int)gc, R, 1, opts->atol, opts->btol, opts->max_iter);
    k_m_update<<<gc, 256, 0, st>>>(rank, L.n_cols, K, VT, W, Y, sc, R, 1, ypart, alive, (int)gs);
    RFM_CUDA_CHECK(cudaGetLastError());
    for (int it = 0; it < opts->max_iter; ++it) {
        if ((rc = fwd()) != RFM_OK) return rc;
        {
            ProfScope ps("k_m_rows", st);
            k_m_rows<<<gr, 256, 0, st>>>(insts, rowlist, T, U, sc, R, part, U32, alive, (int)gs);
        }
        {
            ProfScope ps("k_m_beta", st);
            k_m_beta<<<gs, kMSets * kMSub, 0, st>>>(sc, part, (int)gr, ypart, (int)gc, R, 0, opts->atol, opts->btol, alive);
        }
        if ((rc = trans()) != RFM_OK) return rc;
        {
            ProfScope ps("k_m_cols", st);
            k_m_cols<<<gc, 256, 0, st>>>(rank, L.n_cols, K, Z, VT, sc, R, 0, part, V32, alive, (int)gs);
        }
        {
            ProfScope ps("k_m_alpha", st);
            k_m_alpha<<<gs, kMSets * kMSub, 0, st>>>(sc, part, (int)gc, R, 0, opts->atol, opts->btol, opts->max_iter);
        }
        {
            ProfScope ps("k_m_update", st);
            k_m_update<<<gc, 256, 0, st>>>(rank, L.n_cols, K, VT, W, Y, sc, R, 0, ypart, alive, (int)gs);
        }
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    if (rep) {
        k_m_report<<<gs, 64, 0, st>>>(sc, R, rep);
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    // a_j = S^-1 y_j per right-hand side
    double *out = ws_ptr<double>(mws, M.off_out);
    k_m_out<<<2048, 256, 0, st>>>(Y, L.n_cols, R, out);
    RFM_CUDA_CHECK(cudaGetLastError());
    return launch_coefficients(P, ws, out, A, st, R);
}


}  // namespace rfm
