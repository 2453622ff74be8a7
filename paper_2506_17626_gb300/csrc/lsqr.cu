// lsqr.cu -- LSQR (Paige and Saunders 1982) on the filtered, right-
// preconditioned system of Algorithm 2, for every instance of a system at
// once, in one persistent cooperative launch.
//
// Operator of block b (rows I_b, kept columns r_b):
//   AR64:  Op_b = Ahat_b R_b^-1 (FP64 kept columns, FP64 substitution; Sec. 3.2)
//   Q32 / Q64: Op_b = Q_hat_b (Proposition 3.1), FP32 or FP64 storage
//   PLAIN: Op_b = M_b, all K columns (no filtering, no preconditioner)
// Forward products y = sum_b V_b^T Op_b x_b are formed per block into
// block-row partials t, then summed per global row over the fixed row list.
//
// One iteration = three phases separated by grid barriers:
//   F (blocks): finish the previous iteration's column updates of the block's
//      slots (v = vt/alpha; y += phi/rho w; w = v - theta/rho w) and form
//      t = Op_b v_b;
//   R (rows):   u~ = sum t - alpha u (u = u~/beta kept unnormalised), ||u~||^2;
//   T (blocks): vt = Op_b^T (u~/beta_new) - beta_new v, ||vt||^2.
// The reductions are per-CTA partials in a fixed order, summed by every CTA in
// the same fixed order after the barrier, so every CTA holds bit-identical
// scalars and takes the same stopping decision.  Every barrier wait is bounded
// (globaltimer); on expiry the kernel records RFM_ETIMEOUT and all CTAs leave
// at their next barrier.
#include <cooperative_groups.h>

#include <algorithm>
#include <type_traits>

#include "device.cuh"
#include "prof.cuh"

namespace rfm {

struct LsqrArgs {
    const InstRec *insts;
    const BlkRec *blks;
    int n_blocks, n_inst;
    const void *A;           // operator arena (TA)
    const double *W;         // R_hat (AR64)
    const int32_t *rank;     // kept columns per block (nullptr: all K)
    const int32_t *grow, *rowlist;
    const double *h, *y0;
    double *u, *v, *vt, *w, *y, *t, *part;
    LsqrScal *scal;
    unsigned *bar;           // [0] arrivals, [1] generation, [2] error
    double atol, btol;
    int max_iter;
    uint64_t timeout_ns;
    int64_t n_row_tiles;
    double *snap;            // iterate snapshots (nullable)
    int snap_every, snap_cap;
    int64_t n_cols;
    double *phase_ms;        // per-phase times of CTA 0 (nullable)
    int64_t n_block_rows;
    unsigned long long *bcnt;  // per block: chunks of the transposed product finished (fused products)
    int stall;               // test hook: 1 = the first grid barrier, 2 = the forward tiles' waits never release
    int x_cap;               // staging row length of the forward tiles (>= every rank)
};

constexpr int kThreads = 256;
constexpr int kRowTile = 256;
constexpr int kRowChunk = 4096;     // rows of a block held in shared memory at once
constexpr int kStages = 3;          // bulk-copy ring depth
constexpr int kStageBytes = 20480;  // bytes per ring stage

// ---- bulk asynchronous copies into shared memory, completed on mbarriers ----
__device__ inline unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ inline void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ inline void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ inline void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Waits for the given phase parity of an mbarrier; false after timeout_ns.
__device__ inline bool mbar_wait(uint64_t *bar, unsigned parity, uint64_t timeout_ns) {
    const uint64_t t0 = global_ns();
    unsigned spins = 0;
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if ((++spins & 63u) == 0 && global_ns() - t0 > timeout_ns) return false;
    }
}

// Staging ring in dynamic shared memory (after the scalar state).
struct Ring {
    uint64_t bar[kStages];
    unsigned uses[kStages];
};

// Bounded grid barrier.  Returns false when any CTA has reported an error.
// extra > 0 raises the arrival count that releases it beyond the grid (a
// barrier nothing releases: the test hook of RFM_OPT_LSQR_STALL).
__device__ bool grid_sync(unsigned *bar, uint64_t timeout_ns, unsigned extra = 0) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = bar + 1;
        volatile unsigned *verr = bar + 2;
        unsigned g = *vgen;
        __threadfence();
        unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == gridDim.x - 1 + extra) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            uint64_t t0 = global_ns();
            unsigned spins = 0;
            while (*vgen == g) {
                if (*verr) break;
                __nanosleep(64);
                if ((++spins & 255u) == 0 && global_ns() - t0 > timeout_ns) {
                    atomicCAS(bar + 2, 0u, (unsigned)RFM_ETIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    volatile unsigned *verr = bar + 2;
    return *verr == 0;
}

// Sum of one double over the CTA in a fixed order (result valid in thread 0).
__device__ double cta_sum(double x, double *scratch) {
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[warp] = x;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) s += scratch[w];
    return s;
}

// Back substitution R x = x (R upper r x r, column-major ld, FP64), x in
// shared memory; 32-wide diagonal tiles solved by warp 0 with the tile in
// registers, off-diagonal updates by the whole CTA.
__device__ void tri_solve_upper(const double *__restrict__ R, int ld, int r, double *x) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int nt = (r + 31) / 32;
    for (int T = nt - 1; T >= 0; --T) {
        const int c0 = T * 32, nc = min(32, r - c0);
        if (tid < 32) {
            double row[32];
            const int i = c0 + lane;
#pragma unroll
            for (int j = 0; j < 32; ++j) row[j] = (lane < nc && j < nc) ? R[(int64_t)(c0 + j) * ld + i] : 0.0;
            double xi = lane < nc ? x[i] : 0.0;
#pragma unroll
            for (int j = 31; j >= 0; --j) {
                if (j < nc) {
                    if (lane == j) xi = xi / row[j];
                    double xj = __shfl_sync(0xffffffffu, xi, j);
                    if (lane < j) xi = fma(-row[j], xj, xi);
                }
            }
            if (lane < nc) x[i] = xi;
        }
        __syncthreads();
        for (int i = tid; i < c0; i += kThreads) {
            double s = x[i];
            for (int j = 0; j < nc; ++j) s = fma(-R[(int64_t)(c0 + j) * ld + i], x[c0 + j], s);
            x[i] = s;
        }
        __syncthreads();
    }
}

// Forward substitution R^T x = x.
__device__ void tri_solve_upper_t(const double *__restrict__ R, int ld, int r, double *x) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int nt = (r + 31) / 32;
    for (int T = 0; T < nt; ++T) {
        const int c0 = T * 32, nc = min(32, r - c0);
        if (tid < 32) {
            double col[32];
            const int i = c0 + lane;
#pragma unroll
            for (int j = 0; j < 32; ++j) col[j] = (lane < nc && j < nc) ? R[(int64_t)i * ld + c0 + j] : 0.0;
            double xi = lane < nc ? x[i] : 0.0;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (j < nc) {
                    if (lane == j) xi = xi / col[j];
                    double xj = __shfl_sync(0xffffffffu, xi, j);
                    if (lane > j) xi = fma(-col[j], xj, xi);
                }
            }
            if (lane < nc) x[i] = xi;
        }
        __syncthreads();
        for (int i = c0 + nc + tid; i < r; i += kThreads) {
            double s = x[i];
            const double *Rc = R + (int64_t)i * ld + c0;
            for (int j = 0; j < nc; ++j) s = fma(-Rc[j], x[c0 + j], s);
            x[i] = s;
        }
        __syncthreads();
    }
}

// Per-instance sums of the partial array part[s * G + cta] (same order in
// every CTA).  Warp w reduces instances w, w+8, ...
__device__ void reduce_partials(const double *part, int n_inst, double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, G = gridDim.x;
    for (int s = warp; s < n_inst; s += kThreads / 32) {
        const double *p = part + (int64_t)s * G;
        double x = 0.0;
        for (int c0 = 0; c0 < G; c0 += 32 * 8) {
            double v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {     // all loads in flight before the adds
                const int c = c0 + 32 * k + lane;
                v[k] = c < G ? p[c] : 0.0;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) x += v[k];
        }
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) out[s] = x;
    }
    __syncthreads();
}

// Two reductions of per-CTA partials at once: warps 0-3 take the first
// array's instances, warps 4-7 the second's (each sum in the order of
// reduce_partials).
__device__ void reduce_partials2(const double *pa, double *oa, const double *pb, double *ob, int n_inst) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, G = gridDim.x;
    constexpr int half = kThreads / 64;
    const double *part = warp < half ? pa : pb;
    double *out = warp < half ? oa : ob;
    for (int s = warp % half; s < n_inst; s += half) {
        const double *p = part + (int64_t)s * G;
        double x = 0.0;
        for (int c0 = 0; c0 < G; c0 += 32 * 8) {
            double v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int c = c0 + 32 * k + lane;
                v[k] = c < G ? p[c] : 0.0;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) x += v[k];
        }
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) out[s] = x;
    }
    __syncthreads();
}

template <typename TA>
struct Smem {
    double x[kMaxK];           // block column vector (v, p or z)
    TA xa[kMaxK];              // the same in operator precision
    TA ub[kRowChunk];          // gathered u~ / beta of a row chunk
    double acc[kMaxInst];      // this CTA's per-instance partial sums
    double red[kThreads / 32];
    double tmp[kMaxInst];
    LsqrScal sc[kMaxInst > 64 ? 64 : kMaxInst];
};

template <typename TA, bool TRI>
__global__ void __launch_bounds__(kThreads) k_lsqr(LsqrArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<TA> &S = *reinterpret_cast<Smem<TA> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, G = gridDim.x, cta = blockIdx.x;
    const int ni = a.n_inst;
    const TA *Aop = reinterpret_cast<const TA *>(a.A);
    LsqrScal *sc = S.sc;  // local copy of the scalars (identical in every CTA)
    bool ok = true;

    auto blk_rank = [&](int b) { return a.rank ? a.rank[b] : a.blks[b].K; };
    auto clear_acc = [&]() {
        for (int s = tid; s < ni; s += kThreads) S.acc[s] = 0.0;
        __syncthreads();
    };
    auto flush_acc = [&](int which) {
        __syncthreads();
        for (int s = tid; s < ni; s += kThreads) a.part[((int64_t)which * ni + s) * G + cta] = S.acc[s];
    };

    // ---- staging ring (after Smem<TA> in dynamic shared memory)
    unsigned char *ring_base = smem_raw + ((sizeof(Smem<TA>) + 127) / 128) * 128;
    Ring &RG = *reinterpret_cast<Ring *>(ring_base);
    unsigned char *stage_mem = ring_base + 128;
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&RG.bar[i], 1);
            RG.uses[i] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    // Column chunks of a block: cw columns (contiguous, cw*ldm elements).
    auto chunk_cols = [&](const BlkRec &B) {
        int cw = kStageBytes / (B.ldm * (int)sizeof(TA));
        return cw < 1 ? 1 : cw;
    };
    // Sequence of (block, chunk) of this CTA over the blocks accepted by
    // `take`, streamed through the ring; per block: on_start (uniform), per
    // chunk on_chunk(B, r, c0, nc, tile), at the end on_end(B, r).
    auto stream = [&](auto take, auto on_start, auto on_chunk, auto on_end) {
        // issue cursor
        int ib = cta, ic = 0;
        auto adv_issue = [&]() {
            while (ib < a.n_blocks) {
                const int r = blk_rank(ib);
                if (take(ib) && r > 0) {
                    const int cw = chunk_cols(a.blks[ib]);
                    if (ic * cw < r) return true;
                }
                ib += G;
                ic = 0;
            }
            return false;
        };
        auto issue = [&](int stage) {
            if (!adv_issue()) return;
            if (tid == 0) {
                const BlkRec &B = a.blks[ib];
                const int r = blk_rank(ib), cw = chunk_cols(B);
                const int c0 = ic * cw, nc = min(cw, r - c0);
                const unsigned bytes = (unsigned)(nc * B.ldm * (int)sizeof(TA));
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&RG.bar[stage], bytes);
                bulk_g2s(stage_mem + (size_t)stage * kStageBytes, Aop + B.moff + (int64_t)c0 * B.ldm, bytes,
                         &RG.bar[stage]);
            }
            ++ic;
        };
        for (int st = 0; st < kStages; ++st) issue(st);
        int j = 0;
        for (int b = cta; b < a.n_blocks; b += G) {
            const int r = blk_rank(b);
            if (!take(b) || r <= 0) continue;
            const BlkRec &B = a.blks[b];
            on_start(B, r);
            const int cw = chunk_cols(B);
            for (int c0 = 0; c0 < r; c0 += cw, ++j) {
                const int stage = j % kStages;
                const unsigned par = RG.uses[stage] & 1u;
                if (!mbar_wait(&RG.bar[stage], par, a.timeout_ns)) {
                    if (tid == 0) atomicCAS(a.bar + 2, 0u, (unsigned)RFM_ETIMEOUT);
                }
                const TA *tile = reinterpret_cast<const TA *>(stage_mem + (size_t)stage * kStageBytes);
                on_chunk(B, r, c0, min(cw, r - c0), tile);
                __syncthreads();
                if (tid == 0) RG.uses[stage] += 1;
                __syncthreads();
                issue(stage);
            }
            on_end(B, r);
        }
    };

    // t_b = Op_b x_b for every accepted block; x_b from xsrc (the block's K-slot)
    auto forward_all = [&](auto take, const double *xsrc) {
        // blocks without kept columns contribute zero to their rows
        for (int b = cta; b < a.n_blocks; b += G)
            if (take(b) && blk_rank(b) <= 0)
                for (int i = tid; i < a.blks[b].m; i += kThreads) a.t[a.blks[b].roff + i] = 0.0;
        stream(
            take,
            [&](const BlkRec &B, int r) {
                for (int c = tid; c < r; c += kThreads) S.x[c] = xsrc[B.coff + c];
                __syncthreads();
                if (TRI) tri_solve_upper(a.W + B.moff, B.ldm, r, S.x);
                for (int c = tid; c < r; c += kThreads) S.xa[c] = (TA)S.x[c];
                for (int i = tid; i < B.m; i += kThreads) S.ub[i] = (TA)0;
                __syncthreads();
            },
            [&](const BlkRec &B, int r, int c0, int nc, const TA *tile) {
                for (int i = tid; i < B.m; i += kThreads) {
                    TA s = S.ub[i];
                    int c = 0;
                    for (; c + 4 <= nc; c += 4) {
                        s += tile[(c + 0) * B.ldm + i] * S.xa[c0 + c + 0];
                        s += tile[(c + 1) * B.ldm + i] * S.xa[c0 + c + 1];
                        s += tile[(c + 2) * B.ldm + i] * S.xa[c0 + c + 2];
                        s += tile[(c + 3) * B.ldm + i] * S.xa[c0 + c + 3];
                    }
                    for (; c < nc; ++c) s += tile[c * B.ldm + i] * S.xa[c0 + c];
                    S.ub[i] = s;
                }
            },
            [&](const BlkRec &B, int r) {
                for (int i = tid; i < B.m; i += kThreads) a.t[B.roff + i] = (double)S.ub[i];
                __syncthreads();
            });
    };
    // S.x = Op_b^T (u~ / beta) per accepted block, then on_end(B, r) with it
    auto transpose_all = [&](auto take, auto inv_beta_of, auto on_end) {
        stream(
            take,
            [&](const BlkRec &B, int r) {
                const double ib = inv_beta_of(B);
                for (int i = tid; i < B.m; i += kThreads) S.ub[i] = (TA)(a.u[a.grow[B.roff + i]] * ib);
                __syncthreads();
            },
            [&](const BlkRec &B, int r, int c0, int nc, const TA *tile) {
                for (int c = warp; c < nc; c += kThreads / 32) {
                    const TA *col = tile + c * B.ldm;
                    TA s = (TA)0;
                    for (int i = lane; i < B.m; i += 32) s += col[i] * S.ub[i];
                    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                    if (lane == 0) S.x[c0 + c] = (double)s;
                }
            },
            [&](const BlkRec &B, int r) {
                __syncthreads();
                if (TRI) tri_solve_upper_t(a.W + B.moff, B.ldm, r, S.x);
                on_end(B, r);
            });
    };
    auto all_blocks = [&](int) { return true; };
    auto live_blocks = [&](int b) { return !sc[a.blks[b].inst].done; };

    // ------------------------------------------------------------ init
    for (int s = tid; s < ni && s < 64; s += kThreads) {
        LsqrScal z;
        memset(&z, 0, sizeof(z));
        sc[s] = z;
    }
    __syncthreads();
    // I1: y = y0 or 0, and t = Op P y0 when warm-starting
    for (int b = cta; b < a.n_blocks; b += G) {
        const BlkRec &B = a.blks[b];
        const int r = blk_rank(b), K = B.K;
        for (int c = tid; c < K; c += kThreads) {
            a.y[B.coff + c] = (a.y0 && c < r) ? a.y0[B.coff + c] : 0.0;
            a.w[B.coff + c] = 0.0;
            a.v[B.coff + c] = 0.0;
        }
    }
    __syncthreads();
    if (a.y0) forward_all(all_blocks, a.y);
    __syncthreads();
    ok = grid_sync(a.bar, a.timeout_ns);
    // I2: u~ = h - t-sums, partials of ||u~||^2 (slot 0) and ||h||^2 (slot 1)
    clear_acc();
    __shared__ double hacc[kMaxInst];
    for (int s = tid; s < ni; s += kThreads) hacc[s] = 0.0;
    __syncthreads();
    for (int64_t T = cta; T < a.n_row_tiles; T += G) {
        // map tile to instance
        int s = 0;
        int64_t tcount = 0;
        for (; s < ni; ++s) {
            int64_t nt = (a.insts[s].N + kRowTile - 1) / kRowTile;
            if (T < tcount + nt) break;
            tcount += nt;
        }
        const InstRec &I = a.insts[s];
        const int64_t r = (T - tcount) * kRowTile + tid;
        double uu = 0.0, hh = 0.0;
        if (r < I.N) {
            const int64_t gr = I.row0 + r;
            double acc = 0.0;
            if (a.y0) {
                const int32_t *lst = a.rowlist + I.rl_off + r * I.C;
                for (int e = 0; e < I.C; ++e) {
                    int q = lst[e];
                    if (q >= 0) acc += a.t[q];
                }
            }
            double hv = a.h[gr];
            double uv = hv - acc;
            a.u[gr] = uv;
            uu = uv * uv;
            hh = hv * hv;
        }
        double s1 = cta_sum(uu, S.red);
        double s2 = cta_sum(hh, S.red);
        if (tid == 0) { S.acc[s] += s1; hacc[s] += s2; }
    }
    flush_acc(0);
    for (int s = tid; s < ni; s += kThreads) a.part[((int64_t)1 * ni + s) * G + cta] = hacc[s];
    ok = ok && grid_sync(a.bar, a.timeout_ns);
    if (!ok) return;
    reduce_partials(a.part, ni, S.tmp);
    for (int s = tid; s < ni; s += kThreads) sc[s].beta = sqrt(S.tmp[s]);
    reduce_partials(a.part + (int64_t)ni * G, ni, S.tmp);
    for (int s = tid; s < ni; s += kThreads) sc[s].bnorm = sqrt(S.tmp[s]);
    __syncthreads();
    // a warm start whose residual is not below ||h|| is dropped for a zero
    // start (every CTA takes the same decision from the same sums)
    int back = 0;
    for (int s = tid; s < ni; s += kThreads) {
        sc[s].r0norm = sc[s].beta;
        sc[s].start = a.y0 ? 1 : 0;
        if (a.y0 && !(sc[s].beta < sc[s].bnorm)) {
            sc[s].start = 0;
            sc[s].beta = sc[s].bnorm;
            back = 1;
        }
    }
    back = __syncthreads_or(back);
    if (back) {
        for (int b = cta; b < a.n_blocks; b += G) {
            const BlkRec &B = a.blks[b];
            if (sc[B.inst].start) continue;
            for (int c = tid; c < B.K; c += kThreads) a.y[B.coff + c] = 0.0;
        }
        for (int64_t T = cta; T < a.n_row_tiles; T += G) {
            int s = 0;
            int64_t tcount = 0;
            for (; s < ni; ++s) {
                int64_t nt = (a.insts[s].N + kRowTile - 1) / kRowTile;
                if (T < tcount + nt) break;
                tcount += nt;
            }
            if (sc[s].start) continue;
            const InstRec &I = a.insts[s];
            const int64_t r = (T - tcount) * kRowTile + tid;
            if (r < I.N) a.u[I.row0 + r] = a.h[I.row0 + r];
        }
        ok = grid_sync(a.bar, a.timeout_ns);
        if (!ok) return;
    }
    // I3: vt = Op^T (u~/beta), ||vt||^2
    clear_acc();
    transpose_all(
        all_blocks,
        [&](const BlkRec &B) {
            const double beta = sc[B.inst].beta;
            return beta > 0.0 ? 1.0 / beta : 0.0;
        },
        [&](const BlkRec &B, int r) {
            double part = 0.0;
            for (int c = tid; c < r; c += kThreads) {
                a.vt[B.coff + c] = S.x[c];
                part += S.x[c] * S.x[c];
            }
            double sum = cta_sum(part, S.red);
            if (tid == 0) S.acc[B.inst] += sum;
            __syncthreads();
        });
    flush_acc(2);
    ok = grid_sync(a.bar, a.timeout_ns);
    if (!ok) return;
    reduce_partials(a.part + (int64_t)2 * ni * G, ni, S.tmp);
    for (int s = tid; s < ni; s += kThreads) {
        LsqrScal &q = sc[s];
        q.alpha = sqrt(S.tmp[s]);
        q.phibar = q.beta;
        q.rhobar = q.alpha;
        q.rnorm = q.beta;
        q.arnorm = q.alpha * q.beta;
        q.istop = 7;
        q.itn = 0;
        q.done = (q.beta == 0.0 || q.alpha == 0.0) ? 1 : 0;
        if (q.done) q.istop = 0;
        q.status = 0;
    }
    __syncthreads();

    // ------------------------------------------------------------ loop
    bool first = true;
    for (;;) {
        // F: column updates of the previous iteration, then t = Op v
        clear_acc();
        for (int b = cta; b < a.n_blocks; b += G) {
            const BlkRec &B = a.blks[b];
            const LsqrScal &q = sc[B.inst];
            const int r = blk_rank(b);
            double ypart = 0.0;
            if (!q.done || first) {
                const double ia = q.alpha > 0.0 ? 1.0 / q.alpha : 0.0;
                for (int c = tid; c < r; c += kThreads) {
                    const int64_t o = B.coff + c;
                    const double vn = a.vt[o] * ia;
                    double wv, yv = a.y[o];
                    if (first) {
                        wv = vn;
                    } else {
                        yv = fma(q.phi_rho, a.w[o], yv);
                        wv = fma(-q.theta_rho, a.w[o], vn);
                        a.y[o] = yv;
                        if (a.snap && q.itn % a.snap_every == 0 && q.itn / a.snap_every <= a.snap_cap)
                            a.snap[(int64_t)(q.itn / a.snap_every - 1) * a.n_cols + o] = yv;
                    }
                    a.w[o] = wv;
                    a.v[o] = vn;
                    ypart += yv * yv;
                }
            } else {
                for (int c = tid; c < r; c += kThreads) {
                    double yv = a.y[B.coff + c];
                    ypart += yv * yv;
                }
            }
            double ysum = cta_sum(ypart, S.red);
            if (tid == 0) S.acc[B.inst] += ysum;
            __syncthreads();
        }
        forward_all(live_blocks, a.v);
        flush_acc(0);
        ok = grid_sync(a.bar, a.timeout_ns);
        if (!ok) break;
        // stopping test of the iteration just completed (identical in every CTA)
        reduce_partials(a.part, ni, S.tmp);
        __shared__ int s_all_done;
        if (tid == 0) s_all_done = 1;
        __syncthreads();
        for (int s = tid; s < ni; s += kThreads) {
            LsqrScal &q = sc[s];
            if (q.done) continue;
            q.ynorm = sqrt(S.tmp[s]);
            if (!first) {
                if (q.rnorm <= a.btol * q.bnorm + a.atol * sqrt(q.anorm2) * q.ynorm) { q.done = 1; q.istop = 1; }
                else if (q.arnorm <= a.atol * sqrt(q.anorm2) * q.rnorm) { q.done = 1; q.istop = 2; }
            }
            if (!q.done && q.itn >= a.max_iter) { q.done = 1; q.istop = 7; }
            if (!q.done) { q.itn += 1; atomicAnd(&s_all_done, 0); }
        }
        __syncthreads();
        first = false;
        if (s_all_done) break;
        // R: u~ = sum t - alpha u~/beta
        clear_acc();
        for (int64_t T = cta; T < a.n_row_tiles; T += G) {
            int s = 0;
            int64_t tcount = 0;
            for (; s < ni; ++s) {
                int64_t nt = (a.insts[s].N + kRowTile - 1) / kRowTile;
                if (T < tcount + nt) break;
                tcount += nt;
            }
            const LsqrScal &q = sc[s];
            if (q.done) continue;
            const InstRec &I = a.insts[s];
            const int64_t r = (T - tcount) * kRowTile + tid;
            double uu = 0.0;
            if (r < I.N) {
                const int64_t gr = I.row0 + r;
                const int32_t *lst = a.rowlist + I.rl_off + r * I.C;
                double acc = 0.0;
                for (int e = 0; e < I.C; ++e) {
                    int qq = lst[e];
                    if (qq >= 0) acc += a.t[qq];
                }
                const double ab = q.beta > 0.0 ? q.alpha / q.beta : 0.0;
                double uv = fma(-ab, a.u[gr], acc);
                a.u[gr] = uv;
                uu = uv * uv;
            }
            double s1 = cta_sum(uu, S.red);
            if (tid == 0) S.acc[s] += s1;
        }
        flush_acc(1);
        ok = grid_sync(a.bar, a.timeout_ns);
        if (!ok) break;
        reduce_partials(a.part + (int64_t)ni * G, ni, S.tmp);
        // T: vt = Op^T (u~/beta_new) - beta_new v
        clear_acc();
        transpose_all(
            live_blocks,
            [&](const BlkRec &B) {
                const double bn = sqrt(S.tmp[B.inst]);
                return bn > 0.0 ? 1.0 / bn : 0.0;
            },
            [&](const BlkRec &B, int r) {
                const double bn = sqrt(S.tmp[B.inst]);
                double part = 0.0;
                for (int c = tid; c < r; c += kThreads) {
                    const int64_t o = B.coff + c;
                    double x = fma(-bn, a.v[o], S.x[c]);
                    a.vt[o] = x;
                    part += x * x;
                }
                double sum = cta_sum(part, S.red);
                if (tid == 0) S.acc[B.inst] += sum;
                __syncthreads();
            });
        flush_acc(2);
        ok = grid_sync(a.bar, a.timeout_ns);
        if (!ok) break;
        // plane rotation and estimates (identical in every CTA)
        double *bsum = S.tmp;   // still holds ||u~||^2 per instance
        __shared__ double s_alpha[kMaxInst];
        reduce_partials(a.part + (int64_t)2 * ni * G, ni, s_alpha);
        for (int s = tid; s < ni; s += kThreads) {
            LsqrScal &q = sc[s];
            if (q.done) continue;
            const double beta = sqrt(bsum[s]);
            const double alpha = sqrt(s_alpha[s]);
            q.anorm2 += q.alpha * q.alpha + beta * beta;
            const double rho = sqrt(q.rhobar * q.rhobar + beta * beta);
            const double c = rho > 0.0 ? q.rhobar / rho : 1.0;
            const double sn = rho > 0.0 ? beta / rho : 0.0;
            const double theta = sn * alpha;
            q.rhobar = -c * alpha;
            const double phi = c * q.phibar;
            q.phibar = sn * q.phibar;
            q.phi_rho = rho > 0.0 ? phi / rho : 0.0;
            q.theta_rho = rho > 0.0 ? theta / rho : 0.0;
            q.rnorm = q.phibar;
            q.arnorm = q.phibar * alpha * fabs(c);
            q.c = c;
            q.alpha = alpha;
            q.beta = beta;
            if (!isfinite(q.phibar) || !isfinite(q.rhobar) || !isfinite(q.phi_rho) || !isfinite(q.anorm2)) {
                q.done = 1;
                q.status = RFM_ENUMERIC;
            }
        }
        __syncthreads();
    }
    if (cta == 0) {
        for (int s = tid; s < ni; s += kThreads) {
            const LsqrScal &q = sc[s];
            LsqrScal &o = a.scal[s];
            o = q;
            o.anorm2 = q.anorm2;
        }
    }
}

// a = S^-1 y scattered to the J*K layout with zeros at dropped columns.
__global__ void __launch_bounds__(kThreads) k_coefficients(const BlkRec *__restrict__ blks, const double *__restrict__ W,
                                                           const int32_t *__restrict__ rank,
                                                           const int32_t *__restrict__ perm,
                                                           const double *__restrict__ y, double *__restrict__ out,
                                                           int tri, int64_t set_stride) {
    __shared__ double x[kMaxK];
    const BlkRec &B = blks[blockIdx.x];
    y += blockIdx.y * set_stride;     // data set blockIdx.y of a many-right-hand-side solve
    out += blockIdx.y * set_stride;
    const int r = rank ? rank[blockIdx.x] : B.K;
    for (int c = threadIdx.x; c < B.K; c += kThreads) {
        out[B.coff + c] = 0.0;
        if (c < r) x[c] = y[B.coff + c];
    }
    __syncthreads();
    if (tri) tri_solve_upper(W + B.moff, B.ldm, r, x);
    for (int c = threadIdx.x; c < r; c += kThreads) {
        const int col = perm ? perm[B.coff + c] : c;
        out[B.coff + col] = x[c];
    }
}

// itn_add (nullable): iterations of earlier solves of a refinement, per instance.
__global__ void k_report(const LsqrScal *__restrict__ sc, int n, rfm_lsqr_report *__restrict__ rep, const unsigned *bar,
                         const double *__restrict__ itn_add, const LsqrScal *__restrict__ sc_first) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const LsqrScal &q = sc[s];
    rep[s].itn = q.itn + (itn_add ? itn_add[s] : 0.0);
    rep[s].start = sc_first ? sc_first[s].start : q.start;
    rep[s].r0norm = sc_first ? sc_first[s].r0norm : q.r0norm;
    const double st_now = bar[2] ? (double)bar[2] : (double)q.status;
    const double st_before = itn_add ? itn_add[n + s] : 0.0;
    rep[s].status = st_before != 0.0 ? st_before : st_now;
    rep[s].istop = q.istop;
    rep[s].rnorm = q.rnorm;
    rep[s].arnorm = q.arnorm;
    rep[s].anorm = sqrt(q.anorm2);
    rep[s].ynorm = q.ynorm;
    rep[s].bnorm = q.bnorm;
}


// ---------------------------------------------------------------------------
// Tile variant for the explicit operators (Q_hat in FP32 or FP64, or the
// unfiltered M): the work of every phase is spread over all CTAs, so all SMs
// stream the operator at once.  One iteration = two phases separated by grid
// barriers:
//   rows (R): u~ = (sum of the block partials of each row) / alpha
//     - (alpha/beta) u~, copied onto the block rows in the operator's
//     precision;
//   fused products: one list of warp items holds, per block, its chunks of 8
//     columns (transposed product: z = Op_b^T u~_b, then the FP64 update of
//     vt, y and w per column) and, about 1.2 rounds of the grid's warps
//     later, its 32-row tiles (forward product of the next iteration,
//     t = Op_b vt_b, unscaled); a tile waits on a per-block counter of
//     finished chunks, and re-reads the block while it is still in L2, so
//     the operator comes from DRAM about once per iteration instead of twice.
// Every CTA forms the Givens recurrences redundantly (scalars), in warp 0
// while its other warps issue the row phase's loads.  ||y||^2 rides in the
// fused phase, so the stopping test of iteration i is taken after the fused
// barrier of round i+1 (with iteration i's estimates).
// ---------------------------------------------------------------------------

// Operator loads with an L2 eviction priority (PTX createpolicy + cache_hint):
// a chunk of the transposed product marks its block evict-last, so it is
// still in L2 when the block's forward tiles re-read it; the tiles' loads
// are its last use and mark the lines evict-first.
// Release increment of a completion counter (no returned value to wait for).
__device__ __forceinline__ void red_release_add(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t l2_policy_keep() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_drop() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float4 ld_hint(const float4 *p, uint64_t pol) {
    float4 r;
    asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ double2 ld_hint(const double2 *p, uint64_t pol) {
    double2 r;
    asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;" : "=d"(r.x), "=d"(r.y) : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ float ld_hint(const float *p, uint64_t pol) {
    float r;
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r) : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ double ld_hint(const double *p, uint64_t pol) {
    double r;
    asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r) : "l"(p), "l"(pol));
    return r;
}

static int g_lsqr_stall = 0;
void set_lsqr_stall(int v) { g_lsqr_stall = v; }
static int g_lsqr_lag = 0;   // lag of the fused products' tiles, tenths of a grid round of items (0: automatic)
void set_lsqr_lag(int v) { g_lsqr_lag = v; }

template <typename TA>
struct TileSmem {
    double wacc[2][kThreads / 32][64];          // per-warp partials per instance (alpha^2, ||y||^2)
    double acc_b[64], hacc[64];   // at most 64 instances per solve
    double tmp[64], tmp2[64], yy[64];
    double wred[2][8];
    LsqrScal sc[64];
    // per-instance factors formed once per phase (no division or square root
    // in per-element code: GB300's FP64 pipe is narrow)
    double inv_alpha[64], ab[64], bn[64], inv_bn[64];
    int64_t wt0[65];              // first 32-row warp tile of each instance (row phase)
};

// Four rows of a column owned by one lane: FP32 one 16-byte load of rows
// r0+4l..r0+4l+3; FP64 two 16-byte loads of rows r0+2l, +1 and r0+64+2l, +1.
// Each 16-byte part is loaded only when its first row lies below the column's
// leading dimension ldm (a multiple of 32, so the whole part then does too).
template <typename TA>
struct Rows4;
template <>
struct Rows4<float> {
    __device__ static int row(int r0, int lane, int v) { return r0 + 4 * lane + v; }
    __device__ static void store(float *p, int r0, int lane, int ldm, const float *s) {
        const int i = r0 + 4 * lane;
        if (i < ldm) *reinterpret_cast<float4 *>(p + i) = make_float4(s[0], s[1], s[2], s[3]);
    }
    __device__ static void load_rw(const float *p, int r0, int lane, int ldm, float *q) {
        const int i = r0 + 4 * lane;
        float4 t = i < ldm ? *reinterpret_cast<const float4 *>(p + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        q[0] = t.x; q[1] = t.y; q[2] = t.z; q[3] = t.w;
    }
    __device__ static void load(const float *col, int r0, int lane, int ldm, float *q) {
        const int i = r0 + 4 * lane;
        const bool in = i < ldm;
        float4 t = __ldg(reinterpret_cast<const float4 *>(col + (in ? i : ldm - 4)));   // always a valid address
        q[0] = in ? t.x : 0.f; q[1] = in ? t.y : 0.f; q[2] = in ? t.z : 0.f; q[3] = in ? t.w : 0.f;
    }
};
template <>
struct Rows4<double> {
    __device__ static int row(int r0, int lane, int v) { return r0 + (v < 2 ? 2 * lane + v : 64 + 2 * lane + v - 2); }
    __device__ static void store(double *p, int r0, int lane, int ldm, const double *s) {
        const int i0 = r0 + 2 * lane, i1 = r0 + 64 + 2 * lane;
        if (i0 < ldm) *reinterpret_cast<double2 *>(p + i0) = make_double2(s[0], s[1]);
        if (i1 < ldm) *reinterpret_cast<double2 *>(p + i1) = make_double2(s[2], s[3]);
    }
    __device__ static void load_rw(const double *p, int r0, int lane, int ldm, double *q) {
        const int i0 = r0 + 2 * lane, i1 = r0 + 64 + 2 * lane;
        double2 t0 = i0 < ldm ? *reinterpret_cast<const double2 *>(p + i0) : make_double2(0.0, 0.0);
        double2 t1 = i1 < ldm ? *reinterpret_cast<const double2 *>(p + i1) : make_double2(0.0, 0.0);
        q[0] = t0.x; q[1] = t0.y; q[2] = t1.x; q[3] = t1.y;
    }
    __device__ static void load(const double *col, int r0, int lane, int ldm, double *q) {
        const int i0 = r0 + 2 * lane, i1 = r0 + 64 + 2 * lane;
        const bool in0 = i0 < ldm, in1 = i1 < ldm;
        double2 t0 = __ldg(reinterpret_cast<const double2 *>(col + (in0 ? i0 : ldm - 2)));
        double2 t1 = __ldg(reinterpret_cast<const double2 *>(col + (in1 ? i1 : ldm - 2)));
        q[0] = in0 ? t0.x : 0.0; q[1] = in0 ? t0.y : 0.0;
        q[2] = in1 ? t1.x : 0.0; q[3] = in1 ? t1.y : 0.0;
    }
};

// Live column items in block order: block b contributes ceil(r_b / 8) items.
// One CTA, deterministic prefix sum.
__global__ void __launch_bounds__(1024) k_build_items(const InstRec *__restrict__ insts, int n_inst,
                                                      const BlkRec *__restrict__ blks, int n_blocks,
                                                      const int32_t *__restrict__ rank, ColItem *__restrict__ items,
                                                      int *__restrict__ n_items, ColItem *__restrict__ fitems,
                                                      int *__restrict__ n_fitems, ColItem *__restrict__ titems,
                                                      int *__restrict__ n_titems, int elem_bytes, int64_t t_cap,
                                                      int twarps, int lag_tenths) {
    __shared__ int scan[1024];
    __shared__ int carry;
    const int tid = threadIdx.x;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n_blocks; base += 1024) {
        const int b = base + tid;
        int cnt = 0;
        if (b < n_blocks) {
            const int r = rank ? rank[b] : blks[b].K;
            cnt = (r + kColTile - 1) / kColTile;
        }
        scan[tid] = cnt;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            const int v = tid >= off ? scan[tid - off] : 0;
            __syncthreads();
            scan[tid] += v;
            __syncthreads();
        }
        const int start = carry + scan[tid] - cnt;
        if (b < n_blocks) {
            const BlkRec &B = blks[b];
            const int r = rank ? rank[b] : B.K;
            for (int k = 0; k < cnt; ++k) {
                ColItem it;
                it.b = b;
                it.c0 = k * kColTile;
                it.nc = min(kColTile, r - it.c0);
                it.m = B.m;
                it.ldm = B.ldm;
                it.inst = B.inst;
                it.moff = B.moff;
                it.coff = B.coff;
                it.roff = B.roff;
                items[start + k] = it;
            }
        }
        __syncthreads();
        if (tid == 0) carry += scan[1023];
        __syncthreads();
    }
    if (tid == 0) *n_items = carry;
    // forward items: every 128-row tile of every block with kept columns (nc = r)
    __syncthreads();
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n_blocks; base += 1024) {
        const int b = base + tid;
        int cnt = 0, r = 0;
        if (b < n_blocks) {
            r = rank ? rank[b] : blks[b].K;
            cnt = (blks[b].m + 127) / 128;   // also without kept columns: the tile writes zeros
        }
        scan[tid] = cnt;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            const int v = tid >= off ? scan[tid - off] : 0;
            __syncthreads();
            scan[tid] += v;
            __syncthreads();
        }
        const int start = carry + scan[tid] - cnt;
        if (b < n_blocks) {
            const BlkRec &B = blks[b];
            for (int k = 0; k < cnt; ++k) {
                ColItem it;
                it.b = b;
                it.c0 = k * 128;        // first row of the tile
                it.nc = r;              // kept columns
                it.m = B.m;
                it.ldm = B.ldm;
                it.inst = B.inst;
                it.moff = B.moff;
                it.coff = B.coff;
                it.roff = B.roff;
                fitems[start + k] = it;
            }
        }
        __syncthreads();
        if (tid == 0) carry += scan[1023];
        __syncthreads();
    }
    if (tid == 0) *n_fitems = carry;
    // items of the fused products (transposed product of one round, forward
    // product of the next): block b's column chunks (ceil(r / cc), kind T:
    // nc = columns) and its 32-row tiles (kind F: c0 = first row, nc = -r).
    // A block's tiles need the vector its chunks produce, so they follow its
    // chunks with a lag of L blocks, chosen so that about lag_tenths / 10
    // items per warp of the grid pass in between (1.6 by default): the tiles
    // rarely wait, and the block (re-read by its tiles, kept by an
    // evict-last hint) is still in L2 when the blocks are small enough.
    // Slot s holds the chunks of block s and the tiles of block s - L.
    __shared__ int s_tot;
    __shared__ unsigned long long s_bytes;
    __syncthreads();
    if (tid == 0) {
        s_tot = 0;
        s_bytes = 0ull;
    }
    __syncthreads();
    for (int b = tid; b < n_blocks; b += 1024) {
        const int r = rank ? rank[b] : blks[b].K;
        const int cc = tchunk_cols(blks[b].ldm, elem_bytes);
        atomicAdd(&s_tot, (r + cc - 1) / cc + (blks[b].ldm + 31) / 32);
        atomicAdd(&s_bytes, 2ull * (unsigned long long)blks[b].ldm * (unsigned long long)r * elem_bytes);
    }
    __syncthreads();
    const int tot = s_tot;
    // lag in items: lag_tenths / 10 passes of the grid's warps, or (lag_tenths
    // = 0) that of 1.6 passes capped so that about 120 MB of operator pass
    // between a block's chunks and its tiles (blocks of a few MB need the
    // cap to be re-read from L2; small blocks keep the 1.6 passes)
    int64_t lag_items = (int64_t)twarps * (lag_tenths > 0 ? lag_tenths : 16) / 10;
    if (lag_tenths == 0 && tot > 0 && s_bytes > 0) {
        const double per_item = (double)s_bytes / (double)tot;
        const int64_t cap = (int64_t)(120.0e6 / per_item);
        lag_items = lag_items < cap ? lag_items : (cap > 1 ? cap : 1);
    }
    const int lag = n_blocks > 0 && tot > 0
                        ? (int)min((int64_t)n_blocks, (lag_items * n_blocks + tot - 1) / tot)
                        : 0;
    if (tid == 0) carry = 0;
    __syncthreads();
    const int n_slots = n_blocks + lag;
    for (int base = 0; base < n_slots; base += 1024) {
        const int sl = base + tid;
        int nT = 0, nF = 0, rT = 0, ccT = 1, rF = 0;
        if (sl < n_blocks) {
            rT = rank ? rank[sl] : blks[sl].K;
            ccT = tchunk_cols(blks[sl].ldm, elem_bytes);
            nT = (rT + ccT - 1) / ccT;
        }
        const int bF = sl - lag;
        if (sl < n_slots && bF >= 0) {
            rF = rank ? rank[bF] : blks[bF].K;
            nF = (blks[bF].ldm + 31) / 32;
        }
        const int cnt = nT + nF;
        scan[tid] = cnt;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            const int v = tid >= off ? scan[tid - off] : 0;
            __syncthreads();
            scan[tid] += v;
            __syncthreads();
        }
        const int start = carry + scan[tid] - cnt;
        for (int k = 0; k < nT; ++k) {
            const BlkRec &B = blks[sl];
            ColItem it;
            it.b = sl;
            it.c0 = k * ccT;
            it.nc = min(ccT, rT - it.c0);
            it.m = B.m;
            it.ldm = B.ldm;
            it.inst = B.inst;
            it.moff = B.moff;
            it.coff = B.coff;
            it.roff = B.roff;
            if (start + k < t_cap) titems[start + k] = it;   // the host sizes t_cap for every case
        }
        for (int k = 0; k < nF; ++k) {
            const BlkRec &B = blks[bF];
            ColItem it;
            it.b = bF;
            it.c0 = k * 32;
            it.nc = -rF;
            it.m = B.m;
            it.ldm = B.ldm;
            it.inst = B.inst;
            it.moff = B.moff;
            it.coff = B.coff;
            it.roff = B.roff;
            if (start + nT + k < t_cap) titems[start + nT + k] = it;
        }
        __syncthreads();
        if (tid == 0) carry += scan[1023];
        __syncthreads();
    }
    if (tid == 0) *n_titems = carry < t_cap ? carry : (int)t_cap;
}

template <typename TA>
__global__ void __launch_bounds__(kThreads, 2) k_lsqr_tiles(LsqrArgs a, const ColItem *__restrict__ items,
                                                         const int *__restrict__ n_items_p,
                                                         const ColItem *__restrict__ fitems,
                                                         const int *__restrict__ n_fitems_p, TA *__restrict__ tu,
                                                         const ColItem *__restrict__ titems,
                                                         const int *__restrict__ n_titems_p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem<TA> &S = *reinterpret_cast<TileSmem<TA> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, G = gridDim.x, cta = blockIdx.x;
    const int nwarps = kThreads / 32;
    // worker index: consecutive items go to different CTAs (spread over every SM)
    const int64_t gwarp = (int64_t)warp * G + cta, twarps = (int64_t)G * nwarps;
    const int ni = a.n_inst;
    const int64_t n_items = *n_items_p, n_fitems = *n_fitems_p;
    const TA *Aop = reinterpret_cast<const TA *>(a.A);
    // vt in the operator's precision: the FP64 vector itself, or an FP32 copy
    // in the v arena (unused by this kernel otherwise)
    TA *vx = sizeof(TA) == sizeof(double) ? reinterpret_cast<TA *>(a.vt) : reinterpret_cast<TA *>(a.v);
    LsqrScal *sc = S.sc;
    bool ok = true;
    auto blk_rank = [&](int b) { return a.rank ? __ldg(a.rank + b) : a.blks[b].K; };
    auto clear = [&](double *p) {
        for (int s = tid; s < ni; s += kThreads) p[s] = 0.0;
    };
    auto flush = [&](const double *p, int which) {
        for (int s = tid; s < ni; s += kThreads) a.part[((int64_t)which * ni + s) * G + cta] = p[s];
    };
    auto clear_w = [&]() {
        for (int i = tid; i < 2 * nwarps * 64; i += kThreads) (&S.wacc[0][0][0])[i] = 0.0;
    };
    auto flush_w = [&](int k, int which) {
        for (int s = tid; s < ni; s += kThreads) {
            double t = 0.0;
            for (int w = 0; w < nwarps; ++w) t += S.wacc[k][w][s];
            a.part[((int64_t)which * ni + s) * G + cta] = t;
        }
    };

    // forward items (one warp each): t[rows] = Op_b[rows, :] x_b for a 128-row
    // tile, 8 columns per round trip, x = src * scale(inst)
    auto forward = [&](auto take, const TA *src, auto scale_of) {
        for (int64_t k = gwarp; k < n_fitems; k += twarps) {
            const ColItem it = fitems[k];
            if (!take(it.inst)) continue;
            const double xs = scale_of(it.inst);
            const int r0 = it.c0, r = it.nc;
            const TA *base = Aop + it.moff;
            const TA *xb = src + it.coff;
            TA acc[4] = {(TA)0, (TA)0, (TA)0, (TA)0};
            constexpr int CW = kColTile;   // columns per round trip
            int c = 0;
            for (; c + CW <= r; c += CW) {
                TA q[CW][4];
                TA x[CW];
#pragma unroll
                for (int j = 0; j < CW; ++j) Rows4<TA>::load(base + (int64_t)(c + j) * it.ldm, r0, lane, it.ldm, q[j]);
#pragma unroll
                for (int j = 0; j < CW; ++j) x[j] = xb[c + j];   // written in-kernel: coherent loads
#pragma unroll
                for (int j = 0; j < CW; ++j)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[v] += q[j][v] * x[j];
            }
            for (; c < r; ++c) {
                TA q[4];
                Rows4<TA>::load(base + (int64_t)c * it.ldm, r0, lane, it.ldm, q);
                const TA x = xb[c];
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[v] += q[v] * x;
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int i = Rows4<TA>::row(r0, lane, v);
                if (i < it.m) a.t[it.roff + i] = (double)acc[v] * xs;
            }
        }
    };
    // forward product of block row q (written in this kernel: coherent loads)
    auto row_partials = [&](int64_t q) { return __ldcg(a.t + q); };
    // ---- fused products: the transposed product of a round and the forward
    // product of the next, over one list of warp items (block b's column
    // chunks, then, about 1.2 rounds of the grid later, its 32-row tiles).
    //  chunk (kind T): up to 8 columns of a block; each lane keeps 2 x 8
    //    sixteen-byte operator loads in flight; the 8 column sums are
    //    reduce-scattered in 9 shuffles so that lane 4t holds column t, and
    //    those lanes apply the FP64 epilogue epi (the new vt and its FP32 copy
    //    vx; its FP64 operands were loaded when the chunk started); then the
    //    block's counter of finished chunks is raised (release reduction).
    //  tile (kind F): 32 rows of a block times its r kept columns, t = Op vx
    //    (unscaled: the row phase applies 1/alpha); it waits until every chunk
    //    of the block has finished this phase (bounded wait), stages
    //    the block's vx in shared memory and re-reads the block, which its
    //    chunks have just brought into L2.
    // Per-instance sums ||vt||^2, ||y||^2 stay lane-private until the
    // instance changes.
    const int64_t n_tu = *n_titems_p;
    TA *xs = reinterpret_cast<TA *>(smem_raw + sizeof(TileSmem<TA>)) + (size_t)warp * a.x_cap;
    auto fused = [&](auto take, auto epi, unsigned long long phase) {
        const uint64_t pol_keep = l2_policy_keep(), pol_drop = l2_policy_drop();
        constexpr int VW = sizeof(TA) == 4 ? 4 : 2, STRIP = 32 * VW;
        double pa = 0.0, py = 0.0;
        int cur_inst = -1;
        auto flush_lane = [&]() {
            double x = pa, z = py;
            for (int o = 16; o; o >>= 1) {
                x += __shfl_xor_sync(0xffffffffu, x, o);
                z += __shfl_xor_sync(0xffffffffu, z, o);
            }
            if (lane == 0 && cur_inst >= 0) {
                S.wacc[0][warp][cur_inst] += x;
                S.wacc[1][warp][cur_inst] += z;
            }
            pa = py = 0.0;
        };
        const int mycol = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);   // for lane % 4 == 0
        // static round-robin over the list (the per-warp sums are then the
        // same in every run); the next item's record is fetched while the
        // current one runs.  A tile waits only on chunks earlier in the list,
        // which every warp reaches first, so the earliest waiting tile always
        // finds its chunks running.
        ColItem nxt;
        if (gwarp < n_tu) nxt = titems[gwarp];
        for (int64_t k = gwarp; k < n_tu; k += twarps) {
            const ColItem it = nxt;
            if (k + twarps < n_tu) nxt = titems[k + twarps];
            if (!take(it.inst)) continue;
            if (it.nc <= 0) {
                // ---- forward tile
                const int r = -it.nc;
                if (r > 0) {
                    // every chunk of the block is released once per phase
                    if (lane == 0) {
                        const unsigned long long target =
                            phase * (unsigned long long)((r + kColTile - 1) / kColTile) + (a.stall == 2 ? 1ull : 0ull);
                        volatile unsigned long long *cp = a.bcnt + it.b;
                        const uint64_t t0 = global_ns();
                        unsigned spins = 0;
                        while (*cp < target) {
                            if (*(volatile unsigned *)(a.bar + 2)) break;
                            if ((++spins & 63u) == 0 && global_ns() - t0 > a.timeout_ns) {
                                atomicCAS(a.bar + 2, 0u, (unsigned)RFM_ETIMEOUT);
                                break;
                            }
                        }
                        __threadfence();
                    }
                    __syncwarp();
                    for (int c = lane; c < r; c += 32) xs[c] = __ldcg(vx + it.coff + c);
                    __syncwarp();
                }
                // 8 KB of the block in flight per warp: 64 (FP32) or 32 (FP64)
                // columns of the lane's row per round trip
                constexpr int UF = sizeof(TA) == 4 ? 64 : 32;
                const TA *base = Aop + it.moff + it.c0 + lane;   // row c0 + lane of column 0
                TA acc = (TA)0;
                int c = 0;
                for (; c + UF <= r; c += UF) {
                    TA q[UF];
#pragma unroll
                    for (int j = 0; j < UF; ++j) q[j] = ld_hint(base + (int64_t)(c + j) * it.ldm, pol_drop);
#pragma unroll
                    for (int j = 0; j < UF; ++j) acc += q[j] * xs[c + j];
                }
                for (; c + 8 <= r; c += 8) {
                    TA q[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) q[j] = ld_hint(base + (int64_t)(c + j) * it.ldm, pol_drop);
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc += q[j] * xs[c + j];
                }
                for (; c < r; ++c) acc += ld_hint(base + (int64_t)c * it.ldm, pol_drop) * xs[c];
                a.t[it.roff + it.c0 + lane] = (double)acc;   // rows beyond m are zero padding
                __syncwarp();
                continue;
            }
            // ---- transposed chunk
            if (it.inst != cur_inst) {
                flush_lane();
                cur_inst = it.inst;
            }
            const TA *ub = tu + it.roff;
            const TA *base = Aop + it.moff + (int64_t)it.c0 * it.ldm;
            const int ng = it.nc;
            // the epilogue's lane starts loading its column's FP64 entries now
            const bool elane = (lane & 3) == 0 && mycol < ng;
            const int64_t eo = it.coff + it.c0 + mycol;
            double pre[3] = {0.0, 0.0, 0.0};
            if (elane) {
                pre[0] = __ldcg(a.vt + eo);
                pre[1] = __ldcg(a.w + eo);
                pre[2] = __ldcg(a.y + eo);
            }
            TA acc[8];
#pragma unroll
            for (int cq = 0; cq < 8; ++cq) acc[cq] = (TA)0;
            for (int i0 = 0; i0 < it.ldm; i0 += 2 * STRIP) {
                TA w[2][VW], q[8][2][VW];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int i = i0 + STRIP * h + VW * lane;
                    const bool in = i < it.ldm;
                    if (sizeof(TA) == 4) {
                        const float4 t = in ? *reinterpret_cast<const float4 *>(ub + i) : make_float4(0.f, 0.f, 0.f, 0.f);
                        w[h][0] = (TA)t.x; w[h][1 % VW] = (TA)t.y; w[h][2 % VW] = (TA)t.z; w[h][3 % VW] = (TA)t.w;
                    } else {
                        const double2 t = in ? *reinterpret_cast<const double2 *>(ub + i) : make_double2(0.0, 0.0);
                        w[h][0] = (TA)t.x; w[h][1] = (TA)t.y;
                    }
#pragma unroll
                    for (int cq = 0; cq < 8; ++cq) {
                        const bool ok = in && cq < ng;
                        const TA *src = base + (int64_t)cq * it.ldm + (ok ? i : 0);
                        if (sizeof(TA) == 4) {
                            const float4 t = ok ? ld_hint(reinterpret_cast<const float4 *>(src), pol_keep) : make_float4(0.f, 0.f, 0.f, 0.f);
                            q[cq][h][0] = (TA)t.x; q[cq][h][1 % VW] = (TA)t.y; q[cq][h][2 % VW] = (TA)t.z; q[cq][h][3 % VW] = (TA)t.w;
                        } else {
                            const double2 t = ok ? ld_hint(reinterpret_cast<const double2 *>(src), pol_keep) : make_double2(0.0, 0.0);
                            q[cq][h][0] = (TA)t.x; q[cq][h][1] = (TA)t.y;
                        }
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int cq = 0; cq < 8; ++cq)
#pragma unroll
                        for (int v = 0; v < VW; ++v) acc[cq] += q[cq][h][v] * w[h][v];
            }
            // reduce-scatter: lane 4t ends with the full sum of column t
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const bool hi = lane & 16;
                const TA send = hi ? acc[j] : acc[j + 4], keep = hi ? acc[j + 4] : acc[j];
                acc[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const bool hi = lane & 8;
                const TA send = hi ? acc[j] : acc[j + 2], keep = hi ? acc[j + 2] : acc[j];
                acc[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
            }
            {
                const bool hi = lane & 4;
                const TA send = hi ? acc[0] : acc[1], keep = hi ? acc[1] : acc[0];
                acc[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
            }
            acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 2);
            acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
            if (elane) epi(it.inst, eo, (double)acc[0], pre, &pa, &py);
            // the chunk's columns are written: release them to the block's tiles
            // (__syncwarp orders the lanes' stores before lane 0's release)
            __syncwarp();
            if (lane == 0) red_release_add(a.bcnt + it.b, 1ull);
        }
        flush_lane();
    };

    // rows (R): 32-row warp tiles (a tile never spans two instances), two
    // tiles per warp per pass with their loads issued together; u~ of a row
    // = fn(inst, sum of its block partials, old u~), stored to u and to the
    // row's block-row copies; per-warp, per-instance sums of u~^2 in wacc[0].
    // The loads need no scalars: the first pass's loads are issued before
    // mid() (every thread of the CTA calls it once), where the previous
    // phase's scalars can be formed.
    struct RowPass {
        int si[2], Ci[2];
        bool tv[2], rv[2];
        int64_t gr[2];
        const int32_t *lst[2];
        double acc[2], uo[2];
    };
    auto row_load = [&](RowPass &P, int64_t T0, int64_t tw) {
        const int64_t n_wt = S.wt0[ni];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int64_t T = T0 + (int64_t)j * tw;
            int sx = 0;
            if (T < n_wt)
                while (S.wt0[sx + 1] <= T) ++sx;
            P.si[j] = sx;
            P.tv[j] = T < n_wt;
            const InstRec &I = a.insts[sx];
            const int64_t r = (T - S.wt0[sx]) * 32 + lane;
            P.rv[j] = P.tv[j] && r < I.N;
            P.Ci[j] = I.C;
            P.gr[j] = I.row0 + (P.rv[j] ? r : 0);
            P.lst[j] = a.rowlist + I.rl_off + (P.rv[j] ? r : 0) * I.C;
        }
        P.acc[0] = P.acc[1] = 0.0;
        const int Cm = P.Ci[0] > P.Ci[1] ? P.Ci[0] : P.Ci[1];
        // up to 8 covering blocks: every row-list entry loaded first, then
        // every partial, then the sums in entry order (two round trips
        // instead of two per entry); more: entry by entry
        auto gather = [&](auto cmc) {
            constexpr int CM = decltype(cmc)::value;
            int q0[CM], q1[CM];
            double t0[CM], t1[CM];
#pragma unroll
            for (int e = 0; e < CM; ++e) {
                q0[e] = P.rv[0] && e < P.Ci[0] ? __ldg(P.lst[0] + e) : -1;
                q1[e] = P.rv[1] && e < P.Ci[1] ? __ldg(P.lst[1] + e) : -1;
            }
#pragma unroll
            for (int e = 0; e < CM; ++e) {
                t0[e] = q0[e] >= 0 ? row_partials(q0[e]) : 0.0;
                t1[e] = q1[e] >= 0 ? row_partials(q1[e]) : 0.0;
            }
#pragma unroll
            for (int e = 0; e < CM; ++e) {
                if (q0[e] >= 0) P.acc[0] += t0[e];
                if (q1[e] >= 0) P.acc[1] += t1[e];
            }
        };
        if (Cm <= 1) gather(std::integral_constant<int, 1>{});
        else if (Cm <= 2) gather(std::integral_constant<int, 2>{});
        else if (Cm <= 4) gather(std::integral_constant<int, 4>{});
        else if (Cm <= 8) gather(std::integral_constant<int, 8>{});
        else
            for (int e = 0; e < Cm; ++e) {
                const int q0 = P.rv[0] && e < P.Ci[0] ? P.lst[0][e] : -1;
                const int q1 = P.rv[1] && e < P.Ci[1] ? P.lst[1][e] : -1;
                if (q0 >= 0) P.acc[0] += row_partials(q0);
                if (q1 >= 0) P.acc[1] += row_partials(q1);
            }
#pragma unroll
        for (int j = 0; j < 2; ++j) P.uo[j] = P.rv[j] ? a.u[P.gr[j]] : 0.0;
    };
    auto row_finish = [&](RowPass &P, auto take, auto fn) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (!P.tv[j] || !take(P.si[j])) continue;    // warp-uniform
            double uu = 0.0;
            if (P.rv[j]) {
                const double uv = fn(P.si[j], P.acc[j], P.uo[j]);
                a.u[P.gr[j]] = uv;
                const TA ut = (TA)uv;
                for (int e = 0; e < P.Ci[j]; ++e) {
                    const int q = P.lst[j][e];
                    if (q >= 0) tu[q] = ut;
                }
                uu = uv * uv;
            }
            for (int o = 16; o; o >>= 1) uu += __shfl_xor_sync(0xffffffffu, uu, o);
            if (lane == 0) S.wacc[0][warp][P.si[j]] += uu;
        }
    };
    // part: this warp takes tiles w0, w0 + tw, ...
    auto row_phase = [&](bool part, int64_t w0, int64_t tw, auto take, auto fn, auto mid) {
        const int64_t n_wt = S.wt0[ni];
        RowPass P;
        row_load(P, part ? w0 : n_wt, tw);
        mid();
        if (!part) return;
        row_finish(P, take, fn);
        for (int64_t T0 = w0 + 2 * tw; T0 < n_wt; T0 += 2 * tw) {
            row_load(P, T0, tw);
            row_finish(P, take, fn);
        }
    };

    // elementwise over the kept column slots
    auto each_column = [&](auto take, auto fn) {
        const int64_t total = n_items * kColTile;
        for (int64_t f = (int64_t)cta * kThreads + tid; f < total; f += (int64_t)G * kThreads) {
            const ColItem &it = items[f / kColTile];
            const int j = (int)(f % kColTile);
            if (j >= it.nc || !take(it.inst)) continue;
            fn(it.inst, it.coff + it.c0 + j);
        }
    };
    auto all_inst = [&](int) { return true; };
    auto live = [&](int s) { return !sc[s].done; };
    auto row_tile_inst = [&](int64_t T, int64_t *tcount) {
        int s = 0;
        int64_t tc = 0;
        for (; s < ni; ++s) {
            int64_t nt = (a.insts[s].N + kRowTile - 1) / kRowTile;
            if (T < tc + nt) break;
            tc += nt;
        }
        *tcount = tc;
        return s;
    };

    // ------------------------------------------------------------ init
    for (int s = tid; s < ni; s += kThreads) {
        LsqrScal z;
        memset(&z, 0, sizeof(z));
        sc[s] = z;
    }
    if (tid == 0) {
        int64_t t0 = 0;
        for (int s = 0; s < ni; ++s) {
            S.wt0[s] = t0;
            t0 += (a.insts[s].N + 31) / 32;
        }
        S.wt0[ni] = t0;
    }
    __syncthreads();
    each_column(all_inst, [&](int inst, int64_t o) {
        a.y[o] = a.y0 ? a.y0[o] : 0.0;
        a.w[o] = 0.0;
        if (a.y0) vx[o] = (TA)a.y0[o];   // (FP64: vt holds y0 until the first column phase)
    });
    if (a.y0) {
        ok = grid_sync(a.bar, a.timeout_ns);
        if (!ok) return;
        forward(all_inst, vx, [](int) { return 1.0; });
    }
    ok = grid_sync(a.bar, a.timeout_ns, a.stall == 1 ? 1u : 0u);
    // u~ = h - (Op y0), ||u~||^2, ||h||^2; u~ copied onto the block rows
    clear(S.acc_b);
    clear(S.hacc);
    __syncthreads();
    for (int64_t T = cta; T < a.n_row_tiles; T += G) {
        int64_t tc;
        const int s = row_tile_inst(T, &tc);
        const InstRec &I = a.insts[s];
        const int64_t r = (T - tc) * kRowTile + tid;
        double uu = 0.0, hh = 0.0;
        if (r < I.N) {
            const int64_t gr = I.row0 + r;
            const int32_t *lst = a.rowlist + I.rl_off + r * I.C;
            double acc = 0.0;
            if (a.y0)
                for (int e = 0; e < I.C; ++e) {
                    int q = lst[e];
                    if (q >= 0) acc += row_partials(q);
                }
            const double hv = a.h[gr], uv = hv - acc;
            a.u[gr] = uv;
            for (int e = 0; e < I.C; ++e) {
                int q = lst[e];
                if (q >= 0) tu[q] = (TA)uv;
            }
            uu = uv * uv;
            hh = hv * hv;
        }
        double s1 = cta_sum(uu, S.wred[0]);
        double s2 = cta_sum(hh, S.wred[0]);
        if (tid == 0) { S.acc_b[s] += s1; S.hacc[s] += s2; }
    }
    __syncthreads();
    flush(S.acc_b, 1);
    flush(S.hacc, 0);
    ok = ok && grid_sync(a.bar, a.timeout_ns);
    if (!ok) return;
    reduce_partials(a.part + (int64_t)ni * G, ni, S.tmp);
    reduce_partials(a.part, ni, S.tmp2);
    // a warm start whose residual is not below ||h|| is dropped for a zero
    // start (every CTA takes the same decision from the same sums)
    int back = 0;
    for (int s = tid; s < ni; s += kThreads) {
        const double r0 = sqrt(S.tmp[s]), hn = sqrt(S.tmp2[s]);
        sc[s].r0norm = r0;
        sc[s].bnorm = hn;
        sc[s].start = a.y0 ? 1 : 0;
        if (a.y0 && !(r0 < hn)) {
            sc[s].start = 0;
            back = 1;
        }
        sc[s].beta = sc[s].start ? r0 : hn;
        S.inv_bn[s] = sc[s].beta > 0.0 ? 1.0 / sc[s].beta : 0.0;
    }
    back = __syncthreads_or(back);
    if (back) {
        // those instances restart from zero: y = 0 on their columns, u~ = h on
        // their rows and block rows
        auto fell = [&](int s) { return sc[s].start == 0; };
        each_column(fell, [&](int, int64_t o) { a.y[o] = 0.0; });
        for (int64_t T = cta; T < a.n_row_tiles; T += G) {
            int64_t tc;
            const int s = row_tile_inst(T, &tc);
            if (!fell(s)) continue;
            const InstRec &I = a.insts[s];
            const int64_t r = (T - tc) * kRowTile + tid;
            if (r < I.N) {
                const int64_t gr = I.row0 + r;
                const double hv = a.h[gr];
                a.u[gr] = hv;
                const int32_t *lst = a.rowlist + I.rl_off + r * I.C;
                for (int e = 0; e < I.C; ++e) {
                    const int q = lst[e];
                    if (q >= 0) tu[q] = (TA)hv;
                }
            }
        }
        ok = grid_sync(a.bar, a.timeout_ns);
        if (!ok) return;
    }
    __syncthreads();
    // vt = Op^T u~ / beta, ||vt||^2, fused with t = Op vt (the first loop pass's forward product)
    clear_w();
    __syncthreads();
    unsigned long long fphase = 1;
    fused(all_inst, [&](int inst, int64_t o, double z, const double *pre, double *pa, double *py) {
        const double x = z * S.inv_bn[inst];
        a.vt[o] = x;
        if (sizeof(TA) != sizeof(double)) vx[o] = (TA)x;
        *pa += x * x;
    }, fphase);
    __syncthreads();
    flush_w(0, 2);
    ok = grid_sync(a.bar, a.timeout_ns);
    if (!ok) return;
    reduce_partials(a.part + (int64_t)2 * ni * G, ni, S.tmp);
    for (int s = tid; s < ni; s += kThreads) {
        LsqrScal &q = sc[s];
        q.alpha = sqrt(S.tmp[s]);
        q.phibar = q.beta;
        q.rhobar = q.alpha;
        q.rnorm = q.beta;
        q.arnorm = q.alpha * q.beta;
        q.istop = 7;
        q.itn = 0;
        q.done = (q.beta == 0.0 || q.alpha == 0.0) ? 1 : 0;
        if (q.done) q.istop = 0;
        S.inv_alpha[s] = q.alpha > 0.0 ? 1.0 / q.alpha : 0.0;
        S.ab[s] = q.beta > 0.0 ? q.alpha / q.beta : 0.0;
    }
    __syncthreads();

    // ------------------------------------------------------------ rounds
    // Round n: R forms u~_{n+1} = (Op vt_n) / alpha_n - (alpha_n / beta_n) u~_n
    // from the forward partials of the previous fused phase; the fused phase
    // forms Op^T u~_{n+1}, applies iteration n-1's update of y, w (n = 1:
    // w = v_1), vt_{n+1} = Op^T u~_{n+1} / beta_{n+1} - beta_{n+1} v_n, and the
    // forward partials Op vt_{n+1} of round n+1.  The scalars of round n
    // (test of iteration n-1, rotation of iteration n) are formed by warp 0 of
    // every CTA at the start of round n+1, while warps 1-7 issue the loads of
    // that round's row phase, which only its final combine needs them for.
    uint64_t tph = global_ns();
    double ph[4] = {0.0, 0.0, 0.0, 0.0};
    auto mark = [&](int k) {
        const uint64_t t = global_ns();
        ph[k] += (double)(t - tph) * 1e-6;
        tph = t;
    };
    __shared__ int s_all_done;
    // scalars after the fused phase of round m (warp 0): alpha_{m+1}^2 and
    // ||y_{m-1}||^2 from the CTAs' partials, the test of iteration m-1 and the
    // rotation of iteration m
    auto scalars = [&](int m) {
        for (int s = 0; s < ni; ++s) {
            const double *pa = a.part + ((int64_t)2 * ni + s) * G, *py = a.part + (int64_t)s * G;
            double xa = 0.0, xy = 0.0;
            for (int c0 = 0; c0 < G; c0 += 32 * 8) {
                double va[8], vy[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {   // both arrays' loads in flight before the adds
                    const int c = c0 + 32 * k + lane;
                    va[k] = c < G ? pa[c] : 0.0;
                    vy[k] = c < G ? py[c] : 0.0;
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    xa += va[k];
                    xy += vy[k];
                }
            }
            for (int o = 16; o; o >>= 1) {
                xa += __shfl_xor_sync(0xffffffffu, xa, o);
                xy += __shfl_xor_sync(0xffffffffu, xy, o);
            }
            if (lane == 0) {
                S.tmp2[s] = xa;
                S.yy[s] = xy;
            }
        }
        if (lane == 0) s_all_done = 1;
        __syncwarp();
        const bool firstm = m == 1;
        for (int s = lane; s < ni; s += 32) {
            LsqrScal &q = sc[s];
            if (q.done) continue;
            if (!firstm) {
                // (two square roots and two divisions per iteration: GB300's
                // FP64 pipe makes each one a long serial latency)
                q.ynorm = sqrt(S.yy[s]);
                const double anorm = sqrt(q.anorm2);
                if (q.rnorm <= a.btol * q.bnorm + a.atol * anorm * q.ynorm) { q.done = 1; q.istop = 1; }
                else if (q.arnorm <= a.atol * anorm * q.rnorm) { q.done = 1; q.istop = 2; }
                else if (m - 1 >= a.max_iter) { q.done = 1; q.istop = 7; }
            } else if (a.max_iter == 0) {
                q.done = 1;
                q.istop = 7;
            }
            if (q.done) continue;
            q.itn = m;
            const double beta = S.bn[s];
            const double alpha = sqrt(S.tmp2[s]);
            q.anorm2 += q.alpha * q.alpha + beta * beta;
            const double rho = sqrt(q.rhobar * q.rhobar + beta * beta);
            const double rinv = rho > 0.0 ? 1.0 / rho : 0.0;
            const double c = rho > 0.0 ? q.rhobar * rinv : 1.0;
            const double sn = beta * rinv;
            const double theta = sn * alpha;
            q.rhobar = -c * alpha;
            const double phi = c * q.phibar;
            q.phibar = sn * q.phibar;
            q.phi_rho = phi * rinv;
            q.theta_rho = theta * rinv;
            q.rnorm = q.phibar;
            q.arnorm = q.phibar * alpha * fabs(c);
            q.c = c;
            q.alpha = alpha;
            q.beta = beta;
            S.inv_alpha[s] = alpha > 0.0 ? 1.0 / alpha : 0.0;
            S.ab[s] = alpha * S.inv_bn[s];
            if (!isfinite(q.phibar) || !isfinite(q.rhobar) || !isfinite(q.phi_rho) || !isfinite(q.anorm2)) {
                q.done = 1;
                q.status = RFM_ENUMERIC;
            }
            atomicAnd(&s_all_done, 0);
        }
    };
    const int64_t w7 = (int64_t)(warp - 1) * G + cta, tw7 = (int64_t)(nwarps - 1) * G;
    for (int n = 1;; ++n) {
        const bool first = n == 1;
        // R: u~ = (sum of the block partials) / alpha - (alpha / beta) u~
        clear_w();
        __syncthreads();
        row_phase(warp > 0, w7, tw7, live, [&](int s, double acc, double uo) { return fma(-S.ab[s], uo, acc * S.inv_alpha[s]); },
                  [&]() {
                      if (!first && warp == 0) scalars(n - 1);
                      __syncthreads();
                  });
        if (!first && s_all_done) break;
        __syncthreads();
        flush_w(0, 1);
        ok = grid_sync(a.bar, a.timeout_ns);
        mark(1);
        if (!ok) break;
        reduce_partials(a.part + (int64_t)ni * G, ni, S.tmp);   // beta_{n+1}^2
        for (int s = tid; s < ni; s += kThreads) {
            const double bn = sqrt(S.tmp[s]);
            S.bn[s] = bn;
            S.inv_bn[s] = bn > 0.0 ? 1.0 / bn : 0.0;
        }
        __syncthreads();
        // fused products: vt = Op^T u~ / beta_new - beta_new v_n (after
        // iteration n-1's update of y, w); ||vt||^2; ||y_{n-1}||^2; Op vt
        clear_w();
        __syncthreads();
        ++fphase;
        fused(live, [&](int inst, int64_t o, double z, const double *pre, double *pa, double *py) {
            const LsqrScal &q = sc[inst];
            const double vn = pre[0] * S.inv_alpha[inst];
            double yv = pre[2];
            if (first) {
                a.w[o] = vn;
            } else {
                const double wo = pre[1];
                yv = fma(q.phi_rho, wo, yv);
                a.y[o] = yv;
                a.w[o] = fma(-q.theta_rho, wo, vn);
                if (a.snap && q.itn % a.snap_every == 0 && q.itn / a.snap_every <= a.snap_cap)
                    a.snap[(int64_t)(q.itn / a.snap_every - 1) * a.n_cols + o] = yv;
            }
            const double x = fma(z, S.inv_bn[inst], -S.bn[inst] * vn);
            a.vt[o] = x;
            if (sizeof(TA) != sizeof(double)) vx[o] = (TA)x;
            *pa += x * x;
            *py += yv * yv;
        }, fphase);
        __syncthreads();
        flush_w(0, 2);
        flush_w(1, 0);
        ok = grid_sync(a.bar, a.timeout_ns);
        mark(0);
        if (!ok) break;
    }
    if (cta == 0) {
        for (int s = tid; s < ni; s += kThreads) a.scal[s] = sc[s];
        if (a.phase_ms && tid == 0)
            for (int k = 0; k < 4; ++k) a.phase_ms[k] = ph[k];
    }
}

// ---------------------------------------------------------------------------
// Iterative refinement (Carson and Higham 2018, for the least-squares problem
// of Algorithm 2): the residual r = h - M a of the assembled system in FP64,
// from the stored blocks (FP64, or the FP32 values taken exactly).
// ---------------------------------------------------------------------------

// t[q] = (M_b a_b)(q) for the 32 block rows of one tile, all K columns, FP64
// accumulation: warp w takes columns w, w + 8, ..., lane = row; the eight
// partial sums are added in warp order.
template <typename TM>
__global__ void __launch_bounds__(256) k_block_apply(const BlkRec *__restrict__ blks,
                                                     const int32_t *__restrict__ tile_blk,
                                                     const int32_t *__restrict__ tile_row, const TM *__restrict__ M,
                                                     const double *__restrict__ a, double *__restrict__ t) {
    __shared__ double part[8][33];
    const BlkRec &B = blks[tile_blk[blockIdx.x]];
    const int r0 = tile_row[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const TM *col = M + B.moff + r0 + lane;   // rows r0 + lane < ldm (tiles lie inside the padded block)
    const double *ab = a + B.coff;
    double acc = 0.0;
    for (int c = warp; c < B.K; c += 8) acc = fma((double)__ldg(col + (int64_t)c * B.ldm), __ldg(ab + c), acc);
    part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
        double s = part[0][lane];
        for (int w = 1; w < 8; ++w) s += part[w][lane];
        if (r0 + lane < B.m) t[B.roff + r0 + lane] = s;
    }
}

// r[g] = h[g] - sum over the block rows holding global row g (fixed order).
__global__ void k_residual(const InstRec *__restrict__ insts, int n_inst, const int32_t *__restrict__ rowlist,
                           const double *__restrict__ h, const double *__restrict__ t, double *__restrict__ r,
                           int64_t n_rows) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_rows; g += (int64_t)gridDim.x * blockDim.x) {
        int s = 0;
        while (s + 1 < n_inst && insts[s + 1].row0 <= g) ++s;
        const InstRec &I = insts[s];
        const int32_t *lst = rowlist + I.rl_off + (g - I.row0) * I.C;
        double acc = 0.0;
        for (int e = 0; e < I.C; ++e) {
            const int q = lst[e];
            if (q >= 0) acc += t[q];
        }
        r[g] = h[g] - acc;
    }
}

// out[s * stride] = ||r over the rows of instance s||, one CTA per instance,
// fixed summation order.
__global__ void __launch_bounds__(256) k_inst_norm(const InstRec *__restrict__ insts, const double *__restrict__ r,
                                                   double *__restrict__ out, int stride) {
    __shared__ double red[8];
    const InstRec &I = insts[blockIdx.x];
    double s2 = 0.0;
    for (int64_t i = threadIdx.x; i < I.N; i += 256) s2 = fma(r[I.row0 + i], r[I.row0 + i], s2);
    for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        out[(int64_t)blockIdx.x * stride] = sqrt(t);
    }
}

__global__ void k_add(double *__restrict__ y, const double *__restrict__ d, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += d[i];
}

// acc[s] (+)= itn of the solve just finished; acc[n + s] keeps the first
// nonzero status of the solves so far (a later solve resets the barrier words)
__global__ void k_itn_acc(const LsqrScal *__restrict__ sc, int n, double *__restrict__ acc, int first,
                          const unsigned *__restrict__ bar) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    acc[s] = (first ? 0.0 : acc[s]) + (double)sc[s].itn;
    const double st = bar[2] ? (double)bar[2] : (double)sc[s].status;
    acc[n + s] = (first || acc[n + s] == 0.0) ? st : acc[n + s];
}

static unsigned grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    return (unsigned)(g < 1 ? 1 : (g > 8192 ? 8192 : g));
}

// r = h - M a over every instance; ||r|| per instance to out (nullable) with stride.
static rfm_status residual64(const HostPlan &P, void *ws, const double *a, double *r, double *norm_out, int stride,
                             cudaStream_t st) {
    const Layout &L = P.L;
    double *t = ws_ptr<double>(ws, L.off_t);
    if (L.n_tiles > 0) {
        ProfScope ps("k_block_apply", st);
        const int32_t *tb = ws_ptr<int32_t>(ws, L.off_tile);
        if (L.asm_prec == RFM_ASM_FP32)
            k_block_apply<float><<<(unsigned)L.n_tiles, 256, 0, st>>>(ws_ptr<BlkRec>(ws, L.off_blk), tb,
                                                                       tb + L.n_tiles, ws_ptr<float>(ws, L.off_M), a, t);
        else
            k_block_apply<double><<<(unsigned)L.n_tiles, 256, 0, st>>>(ws_ptr<BlkRec>(ws, L.off_blk), tb,
                                                                        tb + L.n_tiles, ws_ptr<double>(ws, L.off_M), a, t);
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    {
        ProfScope ps("k_residual", st);
        k_residual<<<grid_for(L.n_rows, 256), 256, 0, st>>>(ws_ptr<InstRec>(ws, L.off_inst), L.n_inst,
                                                            ws_ptr<int32_t>(ws, L.off_rowlist),
                                                            ws_ptr<double>(ws, L.off_h), t, r, L.n_rows);
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    if (norm_out) {
        ProfScope ps("k_inst_norm", st);
        k_inst_norm<<<(unsigned)L.n_inst, 256, 0, st>>>(ws_ptr<InstRec>(ws, L.off_inst), r, norm_out, stride);
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    return RFM_OK;
}

rfm_status launch_residual(const HostPlan &P, void *ws, const double *a, double *r_out, double *rnorm,
                           cudaStream_t st) {
    double *r = r_out ? r_out : ws_ptr<double>(ws, P.L.off_rres);
    return residual64(P, ws, a, r, rnorm, 1, st);
}

// a = S^-1 y for nsets vectors n_cols apart (one launch)
rfm_status launch_coefficients(const HostPlan &P, void *ws, const double *y, double *a_out, cudaStream_t st,
                               int nsets) {
    const Layout &L = P.L;
    if (L.n_blocks == 0 || nsets < 1) return RFM_OK;
    const bool plain = L.op == RFM_OP_PLAIN;
    ProfScope ps("k_coefficients", st);
    k_coefficients<<<dim3((unsigned)L.n_blocks, (unsigned)nsets), kThreads, 0, st>>>(
        ws_ptr<BlkRec>(ws, L.off_blk), ws_ptr<double>(ws, L.off_W), plain ? nullptr : ws_ptr<int32_t>(ws, L.off_rank),
        plain ? nullptr : ws_ptr<int32_t>(ws, L.off_perm), y, a_out, plain ? 0 : 1, (int64_t)L.n_cols);
    RFM_CUDA_CHECK(cudaGetLastError());
    return RFM_OK;
}

template <typename TA>
static rfm_status run_lsqr_tiles(const HostPlan &P, void *ws, LsqrArgs &args, cudaStream_t st) {
    int dev = 0, nsm = 0, per = 0;
    RFM_CUDA_CHECK(cudaGetDevice(&dev));
    RFM_CUDA_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const Layout &L = P.L;
    // per warp a staging row of the block vector for the forward tiles
    args.x_cap = (int)(L.n_slots * kColTile);
    const size_t sm = sizeof(TileSmem<TA>) + (size_t)(kThreads / 32) * args.x_cap * sizeof(TA);
    RFM_CUDA_CHECK(cudaFuncSetAttribute(k_lsqr_tiles<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    RFM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_lsqr_tiles<TA>, kThreads, sm));
    if (per < 1) {
        set_error("LSQR kernel does not fit on an SM");
        return RFM_ECUDA;
    }
    int G = nsm * per;
    if (G > kMaxPersistCtas) G = kMaxPersistCtas;
    ColItem *items = ws_ptr<ColItem>(ws, L.off_items);
    int *nitems = ws_ptr<int>(ws, L.off_nitems);
    ColItem *titems = ws_ptr<ColItem>(ws, L.off_titems);
    int *ntitems = ws_ptr<int>(ws, L.off_ntitems);
    {
        ProfScope ps("k_build_items", st);
        k_build_items<<<1, 1024, 0, st>>>(args.insts, args.n_inst, args.blks, args.n_blocks, args.rank, items, nitems,
                                          ws_ptr<ColItem>(ws, L.off_fitems), ws_ptr<int>(ws, L.off_nfitems), titems,
                                          ntitems, (int)sizeof(TA), L.n_t_items, G * (kThreads / 32), g_lsqr_lag);
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    TA *tu = ws_ptr<TA>(ws, L.off_tu);
    // padding block rows of u~ are never written by the row phase: keep them zero
    RFM_CUDA_CHECK(cudaMemsetAsync(tu, 0, sizeof(TA) * (size_t)L.block_rows, st));
    args.bcnt = ws_ptr<unsigned long long>(ws, L.off_bcnt);
    RFM_CUDA_CHECK(cudaMemsetAsync(args.bcnt, 0, sizeof(unsigned long long) * (size_t)L.n_blocks, st));
    const ColItem *citems = items, *cfitems = ws_ptr<ColItem>(ws, L.off_fitems), *ctitems = titems;
    const int *cn = nitems, *cfn = ws_ptr<int>(ws, L.off_nfitems), *ctn = ntitems;
    void *kargs[] = {&args, (void *)&citems, (void *)&cn, (void *)&cfitems, (void *)&cfn, (void *)&tu,
                     (void *)&ctitems, (void *)&ctn};
    ProfScope ps("k_lsqr", st);
    RFM_CUDA_CHECK(cudaLaunchCooperativeKernel((const void *)k_lsqr_tiles<TA>, dim3(G), dim3(kThreads), kargs, sm, st));
    return RFM_OK;
}

template <typename TA, bool TRI>
static rfm_status run_lsqr(const HostPlan &P, void *ws, LsqrArgs &args, cudaStream_t st) {
    int dev = 0, nsm = 0, per = 0;
    RFM_CUDA_CHECK(cudaGetDevice(&dev));
    RFM_CUDA_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const size_t sm = ((sizeof(Smem<TA>) + 127) / 128) * 128 + 128 + (size_t)kStages * kStageBytes;
    // one column of the tallest block must fit in a ring stage, all its rows in the row buffer
    const int64_t ld_max = (P.L.max_m + kLdAlign - 1) / kLdAlign * kLdAlign;
    if (ld_max * (int64_t)sizeof(TA) > kStageBytes || P.L.max_m > kRowChunk) {
        set_error("rfm_lsqr_solve: blocks of %lld rows exceed the LSQR kernel's staging (%d rows)",
                  (long long)P.L.max_m, (int)(kStageBytes / sizeof(TA)));
        return RFM_EINVAL;
    }
    RFM_CUDA_CHECK(cudaFuncSetAttribute(k_lsqr<TA, TRI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    RFM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_lsqr<TA, TRI>, kThreads, sm));
    if (per < 1) {
        set_error("LSQR kernel does not fit on an SM");
        return RFM_ECUDA;
    }
    int G = nsm * per;
    if (G > kMaxPersistCtas) G = kMaxPersistCtas;
    void *kargs[] = {&args};
    ProfScope ps("k_lsqr", st);
    RFM_CUDA_CHECK(cudaLaunchCooperativeKernel((const void *)k_lsqr<TA, TRI>, dim3(G), dim3(kThreads), kargs, sm, st));
    return RFM_OK;
}

static void fill_args(const HostPlan &P, void *ws, const rfm_lsqr_opts *opts, const double *y0, LsqrArgs &A) {
    const Layout &L = P.L;
    memset(&A, 0, sizeof(A));
    A.insts = ws_ptr<InstRec>(ws, L.off_inst);
    A.blks = ws_ptr<BlkRec>(ws, L.off_blk);
    A.n_blocks = (int)L.n_blocks;
    A.n_inst = L.n_inst;
    const bool plain = L.op == RFM_OP_PLAIN;
    A.rank = plain ? nullptr : ws_ptr<int32_t>(ws, L.off_rank);
    A.W = ws_ptr<double>(ws, L.off_W);
    A.grow = ws_ptr<int32_t>(ws, L.off_grow);
    A.rowlist = ws_ptr<int32_t>(ws, L.off_rowlist);
    A.h = ws_ptr<double>(ws, L.off_h);
    A.y0 = y0;
    A.u = ws_ptr<double>(ws, L.off_u);
    A.v = ws_ptr<double>(ws, L.off_v);
    A.vt = ws_ptr<double>(ws, L.off_vt);
    A.w = ws_ptr<double>(ws, L.off_w);
    A.y = ws_ptr<double>(ws, L.off_y);
    A.t = ws_ptr<double>(ws, L.off_t);
    A.part = ws_ptr<double>(ws, L.off_part);
    A.scal = ws_ptr<LsqrScal>(ws, L.off_scal);
    A.bar = ws_ptr<unsigned>(ws, L.off_bar);
    A.atol = opts->atol;
    A.btol = opts->btol;
    A.max_iter = opts->max_iter;
    A.timeout_ns = (uint64_t)(opts->timeout_ms > 0 ? opts->timeout_ms : 10000) * 1000000ull;
    A.stall = g_lsqr_stall;
    int64_t nt = 0;
    for (int s = 0; s < L.n_inst; ++s) nt += (P.inst[s].N + kRowTile - 1) / kRowTile;
    A.n_row_tiles = nt;
    A.n_cols = L.n_cols;
    A.phase_ms = opts->d_phase_ms;
    A.n_block_rows = L.block_rows;
    if (opts->d_snap && opts->snap_every > 0 && opts->snap_cap > 0) {
        A.snap = opts->d_snap;
        A.snap_every = opts->snap_every;
        A.snap_cap = opts->snap_cap;
    }
}

// One LSQR run of the configured operator with the arguments in A.
static rfm_status run_op(const HostPlan &P, void *ws, LsqrArgs &A, cudaStream_t st) {
    const Layout &L = P.L;
    RFM_CUDA_CHECK(cudaMemsetAsync(A.bar, 0, 256, st));
    RFM_CUDA_CHECK(cudaMemsetAsync(A.y, 0, sizeof(double) * L.n_cols, st));   // dropped slots of y read back as 0
    if (L.op == RFM_OP_Q32) {
        A.A = ws_ptr<float>(ws, L.off_q32);
        return run_lsqr_tiles<float>(P, ws, A, st);
    } else if (L.op == RFM_OP_Q64) {
        A.A = ws_ptr<double>(ws, L.off_op);
        return run_lsqr_tiles<double>(P, ws, A, st);
    } else if (L.op == RFM_OP_AR64) {
        A.A = ws_ptr<double>(ws, L.off_op);
        return run_lsqr<double, true>(P, ws, A, st);
    } else if (L.asm_prec == RFM_ASM_FP32) {
        A.A = ws_ptr<float>(ws, L.off_M);
        return run_lsqr_tiles<float>(P, ws, A, st);
    }
    A.A = ws_ptr<double>(ws, L.off_M);
    return run_lsqr_tiles<double>(P, ws, A, st);
}

rfm_status launch_lsqr(const HostPlan &P, void *ws, const rfm_lsqr_opts *opts, const double *y0, double *y_out,
                       double *a_out, rfm_lsqr_report *rep, cudaStream_t st) {
    const Layout &L = P.L;
    if (P.L.n_inst > 64) {
        set_error("rfm_lsqr_solve: at most 64 instances per system");
        return RFM_EINVAL;
    }
    const int R = opts->refine_steps;
    if (R < 0 || R > 64 || opts->refine_iters < 0) {
        set_error("rfm_lsqr_solve: refine_steps must be 0..64 and refine_iters >= 0");
        return RFM_EINVAL;
    }
    LsqrArgs A;
    fill_args(P, ws, opts, y0, A);
    rfm_status rc = run_op(P, ws, A, st);
    if (rc != RFM_OK) return rc;
    const double *y_fin = A.y;
    double *itn_acc = nullptr;
    const LsqrScal *sc0 = nullptr;
    if (R > 0 || opts->d_rnorm64) {
        double *yacc = ws_ptr<double>(ws, L.off_yacc);
        double *r = ws_ptr<double>(ws, L.off_rres);
        double *acc = ws_ptr<double>(ws, L.off_itn);
        LsqrScal *s0 = ws_ptr<LsqrScal>(ws, L.off_scal0);
        RFM_CUDA_CHECK(cudaMemcpyAsync(yacc, A.y, sizeof(double) * L.n_cols, cudaMemcpyDeviceToDevice, st));
        RFM_CUDA_CHECK(cudaMemcpyAsync(s0, A.scal, sizeof(LsqrScal) * L.n_inst, cudaMemcpyDeviceToDevice, st));
        sc0 = s0;
        if (R > 0) itn_acc = acc;
        const unsigned gi = (unsigned)((L.n_inst + 63) / 64);
        for (int s = 0; s <= R; ++s) {
            // after solve s: a = S^-1 y (a_out as scratch), r = h - M a, ||r||
            if (s == R && !opts->d_rnorm64) break;
            rc = launch_coefficients(P, ws, yacc, a_out, st, 1);
            if (rc != RFM_OK) return rc;
            rc = residual64(P, ws, a_out, r, opts->d_rnorm64 ? opts->d_rnorm64 + s : nullptr, R + 1, st);
            if (rc != RFM_OK) return rc;
            if (s == R) break;
            // iterations of solve s, then the correction solve s + 1 from zero on r; y += d
            k_itn_acc<<<gi, 64, 0, st>>>(A.scal, L.n_inst, acc, s == 0, A.bar);
            RFM_CUDA_CHECK(cudaGetLastError());
            rfm_lsqr_opts o = *opts;
            o.max_iter = opts->refine_iters > 0 ? opts->refine_iters : opts->max_iter;
            o.d_snap = nullptr;
            o.d_phase_ms = nullptr;
            fill_args(P, ws, &o, nullptr, A);
            A.h = r;
            rc = run_op(P, ws, A, st);
            if (rc != RFM_OK) return rc;
            ProfScope ps("k_add", st);
            k_add<<<grid_for(L.n_cols, 256), 256, 0, st>>>(yacc, A.y, L.n_cols);
            RFM_CUDA_CHECK(cudaGetLastError());
        }
        y_fin = yacc;
    }
    if (y_out) RFM_CUDA_CHECK(cudaMemcpyAsync(y_out, y_fin, sizeof(double) * L.n_cols, cudaMemcpyDeviceToDevice, st));
    rc = launch_coefficients(P, ws, y_fin, a_out, st, 1);
    if (rc != RFM_OK) return rc;
    if (rep) {
        ProfScope ps("k_report", st);
        k_report<<<(L.n_inst + 63) / 64, 64, 0, st>>>(A.scal, L.n_inst, rep, A.bar, itn_acc, sc0);
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    return RFM_OK;
}

// LSQR from zero on another explicit FP64 operator with the system's block
// structure (the fit of predicted values: its own kept counts, right-hand
// side at the collocation rows); z_out receives the iterate (column slots).
rfm_status launch_lsqr_on(const HostPlan &P, void *ws, const double *Op, const int32_t *rank, const double *rhs,
                          int iters, double *z_out, rfm_lsqr_report *rep, cudaStream_t st) {
    const Layout &L = P.L;
    if (P.L.n_inst > 64) {
        set_error("at most 64 instances per system");
        return RFM_EINVAL;
    }
    rfm_lsqr_opts o;
    memset(&o, 0, sizeof(o));
    o.max_iter = iters;
    o.timeout_ms = 10000;
    LsqrArgs A;
    fill_args(P, ws, &o, nullptr, A);
    A.A = Op;
    A.rank = rank;
    A.h = rhs;
    RFM_CUDA_CHECK(cudaMemsetAsync(A.bar, 0, 256, st));
    rfm_status rc = run_lsqr_tiles<double>(P, ws, A, st);
    if (rc != RFM_OK) return rc;
    RFM_CUDA_CHECK(cudaMemcpyAsync(z_out, A.y, sizeof(double) * L.n_cols, cudaMemcpyDeviceToDevice, st));
    if (rep) {
        ProfScope ps("k_report", st);
        k_report<<<(L.n_inst + 63) / 64, 64, 0, st>>>(A.scal, L.n_inst, rep, A.bar, nullptr, nullptr);
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    return RFM_OK;
}

}  // namespace rfm
