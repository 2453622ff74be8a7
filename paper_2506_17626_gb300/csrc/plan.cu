// plan.cu -- host-side layout of a system: validation, block row sets,
// index tables and the placement of every array in the caller's workspace.
//
// Row sets follow Eq. (6): I_j = {r : w_j(x_r) != 0}, and the window of
// subdomain j is nonzero exactly on the open box |x_i - mu_ji| < sig_ji
// (Sec. 4.2), so membership is decided per dimension by that test on the
// cell-centred grid coordinates.  Because the boxes are equal-width and
// ordered, the points of one subdomain form a contiguous grid-index interval
// along every dimension and the covering subdomains of one point form a
// contiguous subdomain-index interval; both are tabulated here.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace rfm {

static thread_local char g_err[1024];

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

const char *last_error() { return g_err; }

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int nfaces_of(const rfm_problem &p) {
    if (p.hard_bc > 0.0) return 0;   // the ansatz satisfies the boundary condition: no boundary rows
    if (p.pde == RFM_PDE_OSC) return 2;
    return p.pde == RFM_PDE_HEAT ? 2 * (p.dim - 1) + 1 : 2 * p.dim;
}

static int depth_of(const rfm_problem &p) { return p.depth > 1 ? p.depth : 1; }

// Parameters of one subdomain network (the layout of rfm_problem in rfm.h).
static int64_t params_per_subdomain(const rfm_problem &p) {
    const int nl = depth_of(p) > 1 ? p.K : p.dim;
    int64_t c = (int64_t)p.K * (nl + 1);
    int nin = p.dim;
    for (int l = 1; l < depth_of(p); ++l) {
        c += (int64_t)p.K * (nin + 1);
        nin = p.K;
    }
    return c;
}

rfm_status build_plan(const rfm_problem *probs, int n_inst, const rfm_config *cfg, HostPlan *out, char *err,
                      size_t errlen) {
    memset(out, 0, sizeof(*out));
    if (!probs || !cfg || n_inst < 1 || n_inst > kMaxInst) {
        snprintf(err, errlen, "need 1..%d instances and a config", kMaxInst);
        return RFM_EINVAL;
    }
    if (cfg->asm_prec != RFM_ASM_FP64 && cfg->asm_prec != RFM_ASM_FP32) {
        snprintf(err, errlen, "asm_prec must be RFM_ASM_FP64 or RFM_ASM_FP32");
        return RFM_EINVAL;
    }
    if (cfg->op < RFM_OP_AR64 || cfg->op > RFM_OP_PLAIN) {
        snprintf(err, errlen, "unknown operator %d", cfg->op);
        return RFM_EINVAL;
    }
    if (!(cfg->tol >= 0.0) || !(cfg->tol < 1.0)) {
        snprintf(err, errlen, "tol must lie in [0, 1)");
        return RFM_EINVAL;
    }
    std::vector<InstRec> inst(n_inst);
    std::vector<BlkRec> blk;
    std::vector<int32_t> tile_blk, tile_row, cov, fwd_items, col_items;
    int64_t row0 = 0, col0 = 0, prm0 = 0, rl0 = 0, moff = 0, roff = 0, max_m = 0, max_K = 0;

    for (int s = 0; s < n_inst; ++s) {
        const rfm_problem &p = probs[s];
        InstRec &I = inst[s];
        memset(&I, 0, sizeof(I));
        if (p.dim < 1 || p.dim > 3) { snprintf(err, errlen, "instance %d: dim must be 1..3", s); return RFM_EINVAL; }
        if (p.pde != RFM_PDE_POISSON && p.pde != RFM_PDE_HEAT && p.pde != RFM_PDE_OSC) { snprintf(err, errlen, "instance %d: unknown pde", s); return RFM_EINVAL; }
        if (p.pde == RFM_PDE_OSC && (p.dim != 1 || p.family != RFM_FAM_OSC)) { snprintf(err, errlen, "instance %d: the oscillator is one-dimensional with RFM_FAM_OSC", s); return RFM_EINVAL; }
        if (p.family == RFM_FAM_OSC && p.pde != RFM_PDE_OSC) { snprintf(err, errlen, "instance %d: RFM_FAM_OSC needs RFM_PDE_OSC", s); return RFM_EINVAL; }
        if (p.depth < 0 || p.depth > 8) { snprintf(err, errlen, "instance %d: depth must be 0..8", s); return RFM_EINVAL; }
        if (p.depth > 1 && p.K > kMaxDeepK) { snprintf(err, errlen, "instance %d: networks with hidden layers are at most %d wide", s, kMaxDeepK); return RFM_EINVAL; }
        if (p.act < RFM_ACT_TANH || p.act > RFM_ACT_SIN) { snprintf(err, errlen, "instance %d: unknown activation", s); return RFM_EINVAL; }
        if (!(p.hard_bc >= 0.0) || (p.hard_bc > 0.0 && p.pde != RFM_PDE_POISSON)) { snprintf(err, errlen, "instance %d: hard_bc must be >= 0 and is for Poisson problems", s); return RFM_EINVAL; }
        if (p.pde == RFM_PDE_HEAT && p.dim < 2) { snprintf(err, errlen, "instance %d: heat needs dim >= 2", s); return RFM_EINVAL; }
        if (p.K < 1 || p.K > kMaxK) { snprintf(err, errlen, "instance %d: K must be 1..%d", s, kMaxK); return RFM_EINVAL; }
        if (!(p.delta > 0.0)) { snprintf(err, errlen, "instance %d: delta must be > 0", s); return RFM_EINVAL; }
        if (p.family < RFM_FAM_SINPROD || p.family > RFM_FAM_OSC) { snprintf(err, errlen, "instance %d: unknown family", s); return RFM_EINVAL; }
        if (p.family == RFM_FAM_PARAM5 && (p.dim != 2 || p.pde != RFM_PDE_POISSON)) { snprintf(err, errlen, "instance %d: PARAM5 is a 2D Poisson family", s); return RFM_EINVAL; }
        if (p.n_modes < 0 || p.n_modes > 16) { snprintf(err, errlen, "instance %d: n_modes must be 0..16", s); return RFM_EINVAL; }
        int64_t J = 1, NI = 1;
        for (int i = 0; i < p.dim; ++i) {
            if (p.S[i] < 2 || p.S[i] > 4096) { snprintf(err, errlen, "instance %d: S[%d] must be 2..4096", s, i); return RFM_EINVAL; }
            if (p.n[i] < 1 || p.n[i] > (1 << 24)) { snprintf(err, errlen, "instance %d: n[%d] out of range", s, i); return RFM_EINVAL; }
            if (!(p.hi[i] > p.lo[i])) { snprintf(err, errlen, "instance %d: empty box along %d", s, i); return RFM_EINVAL; }
            J *= p.S[i];
            NI *= p.n[i];
        }
        I.dim = p.dim; I.pde = p.pde; I.family = p.family; I.n_modes = p.n_modes;
        I.K = p.K; I.kappa = p.kappa; I.delta = p.delta;
        I.depth = depth_of(p);
        I.act = p.act;
        I.hard_bc = p.hard_bc;
        I.n_prm_sub = params_per_subdomain(p);
        I.n_last = I.depth > 1 ? p.K : p.dim;
        for (int i = 0; i < 3; ++i) {
            I.n[i] = i < p.dim ? p.n[i] : 1;
            I.S[i] = i < p.dim ? p.S[i] : 1;
            I.lo[i] = p.lo[i];
            I.hi[i] = p.hi[i];
        }
        memcpy(I.fam, p.fam, sizeof(I.fam));
        const int nf = nfaces_of(p);
        I.nfaces = nf;
        I.NI = NI;
        int64_t fr = NI, nb_set[2] = {0, 0};
        for (int f = 0; f < nf; ++f) {
            int nd, side;
            face_dims(p.pde, f, &nd, &side);
            int64_t c = 1;
            for (int i = 0; i < p.dim; ++i)
                if (i != nd) c *= p.n[i];
            I.face_row0[f] = fr;
            fr += c;
            nb_set[face_set_of(p.pde, p.dim, f)] += c;
        }
        I.N = fr;
        I.scale_int = 1.0 / sqrt((double)NI);
        for (int l = 0; l < 2; ++l) I.scale_set[l] = nb_set[l] > 0 ? sqrt(p.lam[l] / (double)nb_set[l]) : 0.0;
        I.row0 = row0;
        I.col0 = col0;
        I.prm_off = prm0;
        I.blk0 = (int32_t)blk.size();
        I.nblk = (int32_t)J;

        // per-dimension membership tables
        std::vector<std::vector<int>> box_lo(p.dim), box_n(p.dim), tlo(p.dim), thi(p.dim);
        int C = 1;
        for (int i = 0; i < p.dim; ++i) {
            const int n = p.n[i], S = p.S[i];
            box_lo[i].assign(S, 0);
            box_n[i].assign(S, 0);
            tlo[i].assign(S, 0);
            thi[i].assign(S, 0);
            std::vector<double> xs(n + 2);
            for (int g = 0; g < n; ++g) xs[g] = grid_coord(p.lo[i], p.hi[i], n, g);
            xs[n] = p.lo[i];
            xs[n + 1] = p.hi[i];
            std::vector<int> cfirst(n + 2, -1), ccount(n + 2, 0);
            for (int ji = 0; ji < S; ++ji) {
                double mu, sig;
                sub_geom(p.lo[i], p.hi[i], S, p.delta, ji, &mu, &sig);
                int first = -1, cnt = 0;
                for (int g = 0; g < n + 2; ++g) {
                    if (fabs(xs[g] - mu) < sig) {
                        if (g < n) {
                            if (first < 0) first = g;
                            if (g != first + cnt) { snprintf(err, errlen, "internal: non-contiguous box"); return RFM_EINVAL; }
                            ++cnt;
                        }
                        if (cfirst[g] < 0) cfirst[g] = ji;
                        if (ji != cfirst[g] + ccount[g]) { snprintf(err, errlen, "internal: non-contiguous cover"); return RFM_EINVAL; }
                        ccount[g]++;
                    }
                }
                box_lo[i][ji] = first < 0 ? 0 : first;
                box_n[i][ji] = cnt;
                tlo[i][ji] = fabs(xs[n] - mu) < sig;
                thi[i][ji] = fabs(xs[n + 1] - mu) < sig;
            }
            int mc = 1;
            for (int g = 0; g < n + 2; ++g) mc = ccount[g] > mc ? ccount[g] : mc;
            I.maxcover[i] = mc;
            C *= mc;
            I.cov_off[i] = (int32_t)cov.size();
            for (int g = 0; g < n + 2; ++g) {
                cov.push_back(cfirst[g] < 0 ? 0 : cfirst[g]);
                cov.push_back(ccount[g]);
            }
        }
        for (int i = p.dim; i < 3; ++i) I.maxcover[i] = 1;
        I.C = C;
        I.rl_off = rl0;
        rl0 += I.N * C;

        for (int64_t j = 0; j < J; ++j) {
            BlkRec B;
            memset(&B, 0, sizeof(B));
            B.inst = s;
            B.j = (int32_t)j;
            B.K = p.K;
            int64_t q = j, nint = 1;
            for (int i = 0; i < 3; ++i) {
                if (i < p.dim) {
                    B.jd[i] = (int32_t)(q % p.S[i]);
                    q /= p.S[i];
                    B.box_lo[i] = box_lo[i][B.jd[i]];
                    B.box_n[i] = box_n[i][B.jd[i]];
                    sub_geom(p.lo[i], p.hi[i], p.S[i], p.delta, B.jd[i], &B.mu[i], &B.sig[i]);
                } else {
                    B.jd[i] = 0; B.box_lo[i] = 0; B.box_n[i] = 1; B.mu[i] = 0.0; B.sig[i] = 1.0;
                }
                nint *= B.box_n[i];
            }
            int64_t m = nint;
            for (int f = 0; f < kMaxFaces; ++f) B.face_off[f] = -1;
            for (int f = 0; f < nf; ++f) {
                int nd, side;
                face_dims(p.pde, f, &nd, &side);
                int touch = side ? thi[nd][B.jd[nd]] : tlo[nd][B.jd[nd]];
                int64_t c = 1;
                for (int i = 0; i < p.dim; ++i)
                    if (i != nd) c *= B.box_n[i];
                if (touch && c > 0) {
                    B.face_off[f] = (int32_t)m;
                    m += c;
                }
            }
            if (m == 0) { snprintf(err, errlen, "instance %d: subdomain %lld has no collocation point", s, (long long)j); return RFM_EINVAL; }
            if (m > (1 << 22)) { snprintf(err, errlen, "instance %d: block of %lld rows is too tall", s, (long long)m); return RFM_EINVAL; }
            B.m = (int32_t)m;
            B.n_int = (int32_t)nint;
            B.ldm = (int32_t)((m + kLdAlign - 1) / kLdAlign * kLdAlign);
            B.moff = moff;
            B.roff = roff;
            B.coff = col0 + j * p.K;
            moff += (int64_t)B.ldm * p.K;
            roff += B.ldm;   // block rows at the padded stride: every block starts 128-byte aligned
            max_m = m > max_m ? m : max_m;
            int32_t bi = (int32_t)blk.size();
            for (int64_t r = 0; r < m; r += 32) {
                tile_blk.push_back(bi);
                tile_row.push_back((int32_t)r);
            }
            for (int64_t r = 0; r < m; r += kFwdRows) {
                fwd_items.push_back(bi);
                fwd_items.push_back((int32_t)r);
            }
            for (int c = 0; c < p.K; c += kColTile) {
                col_items.push_back(bi);
                col_items.push_back(c);
            }
            blk.push_back(B);
        }
        max_K = p.K > max_K ? p.K : max_K;
        row0 += I.N;
        col0 += J * p.K;
        prm0 += J * params_per_subdomain(p);
    }

    Layout &L = out->L;
    L.n_inst = n_inst;
    L.n_blocks = (int64_t)blk.size();
    L.n_rows = row0;
    L.n_cols = col0;
    L.block_rows = roff;
    L.max_m = max_m;
    L.max_K = max_K;
    L.n_rowlist = rl0;
    L.n_tiles = (int64_t)tile_blk.size();
    L.n_cov = (int64_t)cov.size();
    L.asm_prec = cfg->asm_prec;
    L.op = cfg->op;
    const size_t melem = (size_t)moff;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
    L.off_inst = take(sizeof(InstRec) * n_inst);
    L.off_blk = take(sizeof(BlkRec) * blk.size());
    L.off_tile = take(sizeof(int32_t) * 2 * tile_blk.size());
    L.off_cov = take(sizeof(int32_t) * (cov.size() + 1));
    L.off_M = take(melem * (cfg->asm_prec == RFM_ASM_FP32 ? 4 : 8));
    L.off_h = take(sizeof(double) * row0);
    L.off_grow = take(sizeof(int32_t) * roff);
    L.off_rowlist = take(sizeof(int32_t) * rl0);
    const bool need_op = cfg->op != RFM_OP_PLAIN;
    L.off_W = take(need_op ? melem * 8 : 0);
    L.off_tau = take(sizeof(double) * col0);
    L.off_perm = take(sizeof(int32_t) * col0);
    L.off_rank = take(sizeof(int32_t) * blk.size());
    L.off_r11 = take(sizeof(double) * blk.size());
    L.off_op = take(need_op ? melem * 8 : 0);
    L.off_q32 = take(cfg->op == RFM_OP_Q32 ? melem * 4 : 0);
    L.off_u = take(sizeof(double) * row0);
    L.off_v = take(sizeof(double) * col0);
    L.off_vt = take(sizeof(double) * col0);
    L.off_w = take(sizeof(double) * col0);
    L.off_y = take(sizeof(double) * col0);
    L.off_t = take(sizeof(double) * roff);
    L.off_part = take(sizeof(double) * 3 * kMaxPersistCtas * n_inst);
    L.off_scal = take(sizeof(LsqrScal) * n_inst);
    L.off_bar = take(256);
    L.off_evpart = take(sizeof(double) * 4 * 1024 * n_inst);
    L.n_prm = prm0;
    L.off_evdf = take(8 * (size_t)(prm0 + col0 + 2));   // double-float copies of the parameters and coefficients
    L.n_fwd_items = (int64_t)fwd_items.size() / 2;
    L.n_col_items = (int64_t)col_items.size() / 2;
    L.off_fwd_items = take(sizeof(int32_t) * (fwd_items.size() + 2));
    L.off_col_items = take(sizeof(int32_t) * (col_items.size() + 2));
    L.n_slots = (max_K + kColTile - 1) / kColTile;
    L.off_items = take(sizeof(ColItem) * (L.n_col_items + 1));
    L.off_nitems = take(256);
    L.off_z = take(sizeof(double) * (col0 + 1));
    {
        // items of the fused products: chunks of the transposed product over
        // every block's K columns and 32-row tiles of the forward product (the
        // ranks are known only on the device; the fit of predicted values runs
        // an FP64 operator on any system)
        int64_t nt = 0;
        for (const BlkRec &B : blk) {
            const int cc = tchunk_cols(B.ldm, 8);
            nt += (B.K + cc - 1) / cc + (B.ldm + 31) / 32;
        }
        L.n_t_items = nt;
    }
    L.off_titems = take(sizeof(ColItem) * (L.n_t_items + 1));
    L.off_ntitems = take(256);
    L.off_bcnt = take(sizeof(unsigned long long) * (blk.size() + 1));
    L.off_qord = take(sizeof(int32_t) * (blk.size() + 1));
    L.off_yacc = take(sizeof(double) * (col0 + 1));
    L.off_rres = take(sizeof(double) * (row0 + 1));
    L.off_itn = take(sizeof(double) * 2 * n_inst);
    L.off_scal0 = take(sizeof(LsqrScal) * n_inst);
    L.off_qblk = take(sizeof(int32_t) * (roff + 1));
    L.off_tu = take(sizeof(double) * (roff + 1));
    L.off_fitems = take(sizeof(ColItem) * (L.n_fwd_items + 1));
    L.off_nfitems = take(256);
    L.total = o;

    out->inst = (InstRec *)malloc(sizeof(InstRec) * n_inst);
    out->blk = (BlkRec *)malloc(sizeof(BlkRec) * (blk.size() + 1));
    out->tile_blk = (int32_t *)malloc(sizeof(int32_t) * 2 * (tile_blk.size() + 1));
    out->tile_row = out->tile_blk + tile_blk.size();
    out->cov = (int32_t *)malloc(sizeof(int32_t) * (cov.size() + 1));
    out->fwd_items = (int32_t *)malloc(sizeof(int32_t) * (fwd_items.size() + 2));
    out->col_items = (int32_t *)malloc(sizeof(int32_t) * (col_items.size() + 2));
    if (!fwd_items.empty()) memcpy(out->fwd_items, fwd_items.data(), sizeof(int32_t) * fwd_items.size());
    if (!col_items.empty()) memcpy(out->col_items, col_items.data(), sizeof(int32_t) * col_items.size());
    memcpy(out->inst, inst.data(), sizeof(InstRec) * n_inst);
    if (!blk.empty()) memcpy(out->blk, blk.data(), sizeof(BlkRec) * blk.size());
    if (!tile_blk.empty()) {
        memcpy(out->tile_blk, tile_blk.data(), sizeof(int32_t) * tile_blk.size());
        memcpy(out->tile_row, tile_row.data(), sizeof(int32_t) * tile_row.size());
    }
    if (!cov.empty()) memcpy(out->cov, cov.data(), sizeof(int32_t) * cov.size());
    // QR launch order: the longest factorizations start first, so that an
    // uneven batch does not end on a few large blocks (longest processing time
    // first); the estimate is the leading term m K min(m, K) of the flops
    out->qr_order = (int32_t *)malloc(sizeof(int32_t) * (blk.size() + 1));
    {
        std::vector<int32_t> ord(blk.size());
        for (size_t b = 0; b < blk.size(); ++b) ord[b] = (int32_t)b;
        auto work = [&](int32_t b) {
            const double m = blk[b].m, k = blk[b].K;
            return m * k * (m < k ? m : k);
        };
        std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return work(a) > work(b); });
        if (!ord.empty()) memcpy(out->qr_order, ord.data(), sizeof(int32_t) * ord.size());
    }
    return RFM_OK;
}

// Global rows (across instances) of block b's rows, in block-row order: the
// index arithmetic of block_row_point (device.cuh) without the coordinates.
void host_block_rows(const HostPlan &P, int64_t b, int64_t *rows) {
    const BlkRec &B = P.blk[b];
    const InstRec &I = P.inst[B.inst];
    for (int lr = 0; lr < B.m; ++lr) {
        int64_t r = 0, stride = 1;
        if (lr < B.n_int) {
            int l = lr;
            for (int i = 0; i < I.dim; ++i) {
                const int g = B.box_lo[i] + l % B.box_n[i];
                l /= B.box_n[i];
                r += g * stride;
                stride *= I.n[i];
            }
        } else {
            int f = -1;
            for (int ff = 0; ff < I.nfaces; ++ff)
                if (B.face_off[ff] >= 0 && B.face_off[ff] <= lr) f = ff;
            int nd, side;
            face_dims(I.pde, f, &nd, &side);
            int l = lr - B.face_off[f];
            r = I.face_row0[f];
            for (int i = 0; i < I.dim; ++i) {
                if (i == nd) continue;
                const int g = B.box_lo[i] + l % B.box_n[i];
                l /= B.box_n[i];
                r += g * stride;
                stride *= I.n[i];
            }
        }
        rows[lr] = I.row0 + r;
    }
}

void free_plan(HostPlan *p) {
    free(p->inst);
    free(p->blk);
    free(p->tile_blk);
    free(p->cov);
    free(p->fwd_items);
    free(p->col_items);
    free(p->qr_order);
    memset(p, 0, sizeof(*p));
}

}  // namespace rfm
