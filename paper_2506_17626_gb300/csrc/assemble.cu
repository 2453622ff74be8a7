// assemble.cu -- block assembly of M and h (Sec. 2.1, Eqs. (1)-(6)).
//
// One CTA per 32-row tile of one block (tiles of all blocks of all instances
// in one launch).  Per row, in FP64: the point, the normalised window and its
// derivatives (product of 1D factors), folded with the row operator and
// weight into coefficients c0, c1, c2 (device.cuh).  Per entry, in the
// assembly precision T: z = b + sum_i w_i (x_i - mu_i)/sig_i, t = tanh(z),
// q = 1 - t^2, and
//   M[r, k] = c0 t + q sum_i a_i (c1_i - 2 a_i t c2_i),  a_i = w_i / sig_i,
// which is the row operator applied to w_j phi_jk (phi' = a q, phi'' = -2 a^2 t q).
// Stores are column-major with 32 consecutive rows per warp (coalesced).
#include "device.cuh"
#include "prof.cuh"

namespace rfm {

__device__ inline float tanh_t(float z) { return tanhf(z); }
__device__ inline double tanh_t(double z) { return tanh(z); }

template <typename T>
__global__ void __launch_bounds__(256) k_assemble(const InstRec *__restrict__ insts, const BlkRec *__restrict__ blks,
                                                  const int32_t *__restrict__ tile_blk,
                                                  const int32_t *__restrict__ tile_row,
                                                  const double *__restrict__ params, T *__restrict__ M) {
    __shared__ double s_x[32][3];
    __shared__ T s_c0[32], s_c1[32][3], s_c2[32][3], s_s[32][3];
    __shared__ BlkRec sB;
    __shared__ InstRec sI;
    const int tile = blockIdx.x;
    if (threadIdx.x == 0) {
        sB = blks[tile_blk[tile]];
        sI = insts[sB.inst];
    }
    __syncthreads();
    const BlkRec &B = sB;
    const InstRec &I = sI;
    const int r0 = tile_row[tile];
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    if (wy == 0) {
        int lr = r0 + lane;
        double c0 = 0.0, c1[3] = {0, 0, 0}, c2[3] = {0, 0, 0}, x[3] = {0, 0, 0};
        if (lr < B.m) {
            int kind, gcov[3];
            block_row_point(I, B, lr, x, &kind, gcov);
            double w, dw[3], d2w[3];
            window_nd(I, B.jd, x, &w, dw, d2w);
            row_coefficients(I, kind, w, dw, d2w, &c0, c1, c2);
        }
        s_c0[lane] = (T)c0;
        for (int i = 0; i < 3; ++i) {
            s_c1[lane][i] = (T)c1[i];
            s_c2[lane][i] = (T)c2[i];
            s_s[lane][i] = (T)(i < I.dim ? (x[i] - B.mu[i]) / B.sig[i] : 0.0);
        }
    }
    __syncthreads();
    const int lr = r0 + lane;
    if (lr >= B.m) {
        // padding rows up to the leading dimension hold zeros
        if (lr < B.ldm)
            for (int k = wy; k < B.K; k += 8) M[B.moff + lr + (int64_t)k * B.ldm] = (T)0;
        return;
    }
    const int d = I.dim;
    const T c0 = s_c0[lane];
    T c1[3], c2[3], sx[3], isg[3];
    for (int i = 0; i < 3; ++i) {
        c1[i] = s_c1[lane][i];
        c2[i] = s_c2[lane][i];
        sx[i] = s_s[lane][i];
        isg[i] = (T)(1.0 / B.sig[i]);
    }
    const double *prm = params + I.prm_off + (int64_t)B.j * I.n_prm_sub;
    T *Mb = M + B.moff + lr;
    if (I.act == RFM_ACT_TANH) {
        for (int k = wy; k < B.K; k += 8) {
            const double *pk = prm + (int64_t)k * (d + 1);
            T z = (T)pk[d];
            T wv[3], a[3];
            for (int i = 0; i < 3; ++i) {
                wv[i] = i < d ? (T)pk[i] : (T)0;
                z += wv[i] * sx[i];
                a[i] = wv[i] * isg[i];
            }
            T t = tanh_t(z);
            T q = (T)1 - t * t;
            T acc = (T)0;
            for (int i = 0; i < 3; ++i) acc += a[i] * (c1[i] - (T)2 * a[i] * t * c2[i]);
            Mb[(int64_t)k * B.ldm] = c0 * t + q * acc;
        }
        return;
    }
    // other activations: phi = Xi(z), dphi/dx_i = Xi'(z) a_i, d2phi/dx_i^2 = Xi''(z) a_i^2
    for (int k = wy; k < B.K; k += 8) {
        const double *pk = prm + (int64_t)k * (d + 1);
        T z = (T)pk[d];
        T a[3];
        for (int i = 0; i < 3; ++i) {
            const T wv = i < d ? (T)pk[i] : (T)0;
            z += wv * sx[i];
            a[i] = wv * isg[i];
        }
        T f, f1, f2;
        act_eval(I.act, z, &f, &f1, &f2);
        T acc = (T)0;
        for (int i = 0; i < 3; ++i) acc += a[i] * (c1[i] * f1 + c2[i] * a[i] * f2);
        Mb[(int64_t)k * B.ldm] = c0 * f + acc;
    }
}

// Networks with hidden layers (Eq. (2), depth h > 1, K <= kMaxDeepK): one CTA
// per 32-row tile as above; warp 0 forms, per row, the row coefficients and
// the output layer's input z with its partial derivatives (FP64 forward
// propagation through the hidden layers, net_hidden) into shared memory;
// then every warp takes features k = warp, warp + 8, ...: s = w_k . z + b_k,
// ds_i = w_k . dz_i, d2s_i = w_k . d2z_i, and
//   M[r, k] = c0 Xi(s) + sum_i c1_i Xi'(s) ds_i + c2_i (Xi''(s) ds_i^2 + Xi'(s) d2s_i).
// FP64 throughout (the assembly precision only at the store).
template <typename T>
__global__ void __launch_bounds__(256) k_assemble_deep(const InstRec *__restrict__ insts,
                                                       const BlkRec *__restrict__ blks,
                                                       const int32_t *__restrict__ tile_blk,
                                                       const int32_t *__restrict__ tile_row,
                                                       const double *__restrict__ params, T *__restrict__ M) {
    extern __shared__ double s_deep[];   // per row: z, dz (3 x kMaxDeepK), d2z (3 x kMaxDeepK)
    double(*s_z)[kMaxDeepK] = reinterpret_cast<double(*)[kMaxDeepK]>(s_deep);
    double(*s_dz)[3 * kMaxDeepK] = reinterpret_cast<double(*)[3 * kMaxDeepK]>(s_deep + 32 * kMaxDeepK);
    double(*s_d2z)[3 * kMaxDeepK] = reinterpret_cast<double(*)[3 * kMaxDeepK]>(s_deep + 32 * 4 * kMaxDeepK);
    __shared__ double s_c0[32], s_c1[32][3], s_c2[32][3];
    __shared__ BlkRec sB;
    __shared__ InstRec sI;
    const int tile = blockIdx.x;
    if (threadIdx.x == 0) {
        sB = blks[tile_blk[tile]];
        sI = insts[sB.inst];
    }
    __syncthreads();
    const BlkRec &B = sB;
    const InstRec &I = sI;
    const int r0 = tile_row[tile];
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const double *prm = params + I.prm_off + (int64_t)B.j * I.n_prm_sub;
    if (wy == 0) {
        const int lr = r0 + lane;
        double c0 = 0.0, c1[3] = {0, 0, 0}, c2[3] = {0, 0, 0}, x[3] = {0, 0, 0};
        if (lr < B.m) {
            int kind, gcov[3];
            block_row_point(I, B, lr, x, &kind, gcov);
            double w, dw[3], d2w[3];
            window_nd(I, B.jd, x, &w, dw, d2w);
            row_coefficients(I, kind, w, dw, d2w, &c0, c1, c2);
            double xn[3], isg[3];
            for (int i = 0; i < 3; ++i) {
                xn[i] = i < I.dim ? (x[i] - B.mu[i]) / B.sig[i] : 0.0;
                isg[i] = 1.0 / B.sig[i];
            }
            net_hidden(I, prm, xn, isg, s_z[lane], s_dz[lane], s_d2z[lane]);
        }
        s_c0[lane] = c0;
        for (int i = 0; i < 3; ++i) {
            s_c1[lane][i] = c1[i];
            s_c2[lane][i] = c2[i];
        }
    }
    __syncthreads();
    const int lr = r0 + lane;
    if (lr >= B.m) {
        if (lr < B.ldm)
            for (int k = wy; k < B.K; k += 8) M[B.moff + lr + (int64_t)k * B.ldm] = (T)0;
        return;
    }
    const int d = I.dim, nin = I.n_last;
    T *Mb = M + B.moff + lr;
    for (int k = wy; k < B.K; k += 8) {
        const double *pk = prm + (int64_t)k * (nin + 1);
        double sv = pk[nin], ds[3] = {0, 0, 0}, d2s[3] = {0, 0, 0};
        for (int m = 0; m < nin; ++m) {
            sv = fma(pk[m], s_z[lane][m], sv);
            for (int i = 0; i < d; ++i) {
                ds[i] = fma(pk[m], s_dz[lane][i * kMaxDeepK + m], ds[i]);
                d2s[i] = fma(pk[m], s_d2z[lane][i * kMaxDeepK + m], d2s[i]);
            }
        }
        double f, f1, f2;
        act_eval(I.act, sv, &f, &f1, &f2);
        double v = s_c0[lane] * f;
        for (int i = 0; i < d; ++i) v += s_c1[lane][i] * f1 * ds[i] + s_c2[lane][i] * (f2 * ds[i] * ds[i] + f1 * d2s[i]);
        Mb[(int64_t)k * B.ldm] = (T)v;
    }
}

// Row maps: grow[q] (global row of block row q) and, per global row, the list
// of block rows that cover it at a fixed position (mixed radix over the
// covering subdomain offsets per dimension), so that sums over a row's blocks
// run in a fixed order.
__global__ void __launch_bounds__(32) k_rowmap(const InstRec *__restrict__ insts, const BlkRec *__restrict__ blks,
                                               const int32_t *__restrict__ tile_blk,
                                               const int32_t *__restrict__ tile_row,
                                               const int32_t *__restrict__ cov, int32_t *__restrict__ grow,
                                               int32_t *__restrict__ rowlist, int32_t *__restrict__ qblk) {
    const int tile = blockIdx.x;
    const BlkRec &B = blks[tile_blk[tile]];
    const InstRec &I = insts[B.inst];
    const int lr = tile_row[tile] + threadIdx.x;
    if (lr >= B.m) return;
    double x[3];
    int kind, gcov[3];
    int64_t r = block_row_point(I, B, lr, x, &kind, gcov);
    int64_t e = 0, rad = 1;
    for (int i = 0; i < I.dim; ++i) {
        int first = cov[I.cov_off[i] + 2 * gcov[i]];
        e += (int64_t)(B.jd[i] - first) * rad;
        rad *= I.maxcover[i];
    }
    const int64_t q = B.roff + lr;
    grow[q] = (int32_t)(I.row0 + r);
    qblk[q] = tile_blk[tile];
    rowlist[I.rl_off + r * I.C + e] = (int32_t)q;
}

// h = [f / sqrt(N_I); sqrt(lam_l / N_B^(l)) g] over the rows of one instance.
__global__ void k_rhs(const InstRec *__restrict__ insts, int s, double *__restrict__ h) {
    const InstRec &I = insts[s];
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < I.N; r += (int64_t)gridDim.x * blockDim.x) {
        double x[3];
        int kind;
        row_point(I, r, x, &kind);
        h[I.row0 + r] = kind < 0 ? I.scale_int * fam_source(I, x) : I.scale_set[kind] * fam_bdata(I, x, kind);
    }
}

// h of every data set of a family sharing one row layout: recs[j] is the
// record of set j (rows from 0), uploaded into the first bytes of scratch
// (room for R records); H[j * N + r].
rfm_status launch_rhs_many(const InstRec *recs, int R, int64_t N, double *H, void *scratch, cudaStream_t st) {
    InstRec *d = reinterpret_cast<InstRec *>(scratch);
    RFM_CUDA_CHECK(cudaMemcpyAsync(d, recs, sizeof(InstRec) * R, cudaMemcpyHostToDevice, st));
    unsigned g = (unsigned)((N + 255) / 256);
    g = g > 4096 ? 4096 : (g < 1 ? 1 : g);
    for (int j = 0; j < R; ++j) {
        ProfScope ps("k_rhs", st);
        k_rhs<<<g, 256, 0, st>>>(d, j, H + (int64_t)j * N);
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    return RFM_OK;
}

rfm_status launch_assemble(const HostPlan &P, void *ws, const double *params, cudaStream_t st) {
    const Layout &L = P.L;
    InstRec *dI = ws_ptr<InstRec>(ws, L.off_inst);
    BlkRec *dB = ws_ptr<BlkRec>(ws, L.off_blk);
    int32_t *dTB = ws_ptr<int32_t>(ws, L.off_tile);
    int32_t *dTR = dTB + L.n_tiles;
    int32_t *dCov = ws_ptr<int32_t>(ws, L.off_cov);
    RFM_CUDA_CHECK(cudaMemsetAsync(ws_ptr<int32_t>(ws, L.off_rowlist), 0xff, sizeof(int32_t) * L.n_rowlist, st));
    if (L.n_tiles > 0) {
        { ProfScope ps("k_rowmap", st);
        k_rowmap<<<(unsigned)L.n_tiles, 32, 0, st>>>(dI, dB, dTB, dTR, dCov, ws_ptr<int32_t>(ws, L.off_grow),
                                                      ws_ptr<int32_t>(ws, L.off_rowlist),
                                                      ws_ptr<int32_t>(ws, L.off_qblk)); }
        RFM_CUDA_CHECK(cudaGetLastError());
        ProfScope ps("k_assemble", st);
        bool deep = false;
        for (int s = 0; s < L.n_inst; ++s) deep = deep || P.inst[s].depth > 1;
        // one launch over every tile; a system with any deep network takes the
        // deep kernel for all its tiles (it also computes one-layer networks:
        // their output-layer input is the normalised point)
        if (deep) {
            const int sm = (int)(sizeof(double) * 32 * 7 * kMaxDeepK);
            if (L.asm_prec == RFM_ASM_FP32) {
                RFM_CUDA_CHECK(cudaFuncSetAttribute(k_assemble_deep<float>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
                k_assemble_deep<float><<<(unsigned)L.n_tiles, 256, sm, st>>>(dI, dB, dTB, dTR, params,
                                                                              ws_ptr<float>(ws, L.off_M));
            } else {
                RFM_CUDA_CHECK(cudaFuncSetAttribute(k_assemble_deep<double>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
                k_assemble_deep<double><<<(unsigned)L.n_tiles, 256, sm, st>>>(dI, dB, dTB, dTR, params,
                                                                               ws_ptr<double>(ws, L.off_M));
            }
        } else if (L.asm_prec == RFM_ASM_FP32) {
            k_assemble<float><<<(unsigned)L.n_tiles, 256, 0, st>>>(dI, dB, dTB, dTR, params, ws_ptr<float>(ws, L.off_M));
        } else {
            k_assemble<double><<<(unsigned)L.n_tiles, 256, 0, st>>>(dI, dB, dTB, dTR, params, ws_ptr<double>(ws, L.off_M));
        }
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    for (int s = 0; s < L.n_inst; ++s) {
        int64_t N = P.inst[s].N;
        unsigned g = (unsigned)((N + 255) / 256);
        g = g > 4096 ? 4096 : (g < 1 ? 1 : g);
        ProfScope ps("k_rhs", st);
        k_rhs<<<g, 256, 0, st>>>(dI, s, ws_ptr<double>(ws, L.off_h));
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    return RFM_OK;
}

}  // namespace rfm
