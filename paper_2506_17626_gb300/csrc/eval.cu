// eval.cu -- the ansatz of Eq. (1) at query points and the error sums of
// Sec. 4.2 (relative L2 and the normalised L1 error e_L1).
//
// One warp per point: the covering subdomains along each dimension are found
// from the box test around the nearest centre; for every covering subdomain
// the lanes split the K features (sum_k a_jk tanh(...)), the sum is weighted
// by the normalised window (product of 1D factors) and reduced in the warp.
// Error sums are reduced per CTA in a fixed order, then per instance.
// The per-feature work (the argument and tanh of every feature at every
// point, about 470 per point in 2D) runs in double-float arithmetic on the
// FP32 pipe (GB300 issues FP64 at 1/64 of the FP32 rate) from double-float
// copies of the parameters and coefficients made once per call; windows,
// the exact solution and the sums stay in FP64.
#include "df.cuh"
#include "device.cuh"
#include "prof.cuh"

namespace rfm {

constexpr int kEvalCtas = 1024;

__global__ void __launch_bounds__(256) k_eval(const InstRec *__restrict__ insts, int s, const double *__restrict__ params,
                                              const double *__restrict__ a, const double *__restrict__ X, int64_t npts,
                                              double *__restrict__ u_out, double *__restrict__ part) {
    const InstRec &I = insts[s];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ double red[8][4];
    double e2 = 0.0, u2 = 0.0, e1 = 0.0, u1 = 0.0;
    const int d = I.dim;
    for (int64_t p = (int64_t)blockIdx.x * 8 + warp; p < npts; p += (int64_t)gridDim.x * 8) {
        double x[3] = {X[3 * p], X[3 * p + 1], X[3 * p + 2]};
        int jlo[3] = {0, 0, 0}, jn[3] = {1, 1, 1};
        for (int i = 0; i < d; ++i) {
            const double sp = (I.hi[i] - I.lo[i]) / (double)(I.S[i] - 1);
            int c = (int)floor((x[i] - I.lo[i]) / sp + 0.5);
            const int H = (int)ceil(I.delta) + 1;
            int a0 = c - H < 0 ? 0 : c - H, a1 = c + H > I.S[i] - 1 ? I.S[i] - 1 : c + H;
            int first = -1, cnt = 0;
            for (int l = a0; l <= a1; ++l) {
                double mu, sig;
                sub_geom(I.lo[i], I.hi[i], I.S[i], I.delta, l, &mu, &sig);
                if (fabs(x[i] - mu) < sig) {
                    if (first < 0) first = l;
                    ++cnt;
                }
            }
            jlo[i] = first < 0 ? 0 : first;
            jn[i] = cnt;
        }
        double uh = 0.0;
        const int ncomb = jn[0] * jn[1] * jn[2];
        for (int cmb = 0; cmb < ncomb; ++cmb) {
            int jd[3], q = cmb;
            int64_t j = 0, stride = 1;
            for (int i = 0; i < 3; ++i) {
                jd[i] = jlo[i] + q % jn[i];
                q /= jn[i];
                if (i < d) {
                    j += jd[i] * stride;
                    stride *= I.S[i];
                }
            }
            double mu[3] = {0, 0, 0}, sig[3] = {1, 1, 1};
            for (int i = 0; i < d; ++i) sub_geom(I.lo[i], I.hi[i], I.S[i], I.delta, jd[i], &mu[i], &sig[i]);
            const double *prm = params + I.prm_off + j * I.n_prm_sub;
            const double *aj = a + I.col0 + j * I.K;
            double sj = 0.0;
            if (I.depth > 1) {
                // the output layer's input: the last hidden layer at the point (Eq. (2))
                double xn[3] = {0, 0, 0}, isg[3] = {1, 1, 1}, z[kMaxDeepK];
                for (int i = 0; i < d; ++i) xn[i] = (x[i] - mu[i]) / sig[i];
                net_hidden(I, prm, xn, isg, z, nullptr, nullptr);
                const int nin = I.n_last;
                for (int k = lane; k < I.K; k += 32) {
                    const double *pk = prm + (int64_t)k * (nin + 1);
                    double sv = pk[nin];
                    for (int m = 0; m < nin; ++m) sv = fma(pk[m], z[m], sv);
                    double f, f1, f2;
                    act_eval(I.act, sv, &f, &f1, &f2);
                    sj = fma(aj[k], f, sj);
                }
            } else {
                for (int k = lane; k < I.K; k += 32) {
                    const double *pk = prm + (int64_t)k * (d + 1);
                    double z = pk[d];
                    for (int i = 0; i < d; ++i) z += pk[i] * ((x[i] - mu[i]) / sig[i]);
                    double f = 0.0;
                    if (I.act == RFM_ACT_TANH) {
                        f = tanh(z);
                    } else {
                        double f1, f2;
                        act_eval(I.act, z, &f, &f1, &f2);
                    }
                    sj = fma(aj[k], f, sj);
                }
            }
            for (int o = 16; o; o >>= 1) sj += __shfl_xor_sync(0xffffffffu, sj, o);
            double w, dw[3], d2w[3];
            window_nd(I, jd, x, &w, dw, d2w);
            uh = fma(w, sj, uh);
        }
        if (lane == 0) {
            u_out[p] = uh;
            const double ue = fam_exact(I, x);
            const double df = uh - ue;
            e2 += df * df;
            u2 += ue * ue;
            e1 += fabs(df);
            u1 += ue;
        }
    }
    if (lane == 0) {
        red[warp][0] = e2; red[warp][1] = u2; red[warp][2] = e1; red[warp][3] = u1;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w][threadIdx.x];
        part[((int64_t)s * kEvalCtas + blockIdx.x) * 4 + threadIdx.x] = t;
    }
}

// double-float copies of the feature parameters (prm0 doubles) and of a (n_cols)
__global__ void k_eval_split(const double *__restrict__ params, int64_t n_prm, const double *__restrict__ a,
                             int64_t n_cols, float2 *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_prm + n_cols;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = df_from_double(i < n_prm ? params[i] : a[i - n_prm]);
}

__global__ void __launch_bounds__(256) k_eval_df(const InstRec *__restrict__ insts, int s,
                                                 const float2 *__restrict__ prm_df, const float2 *__restrict__ a_df,
                                                 const double *__restrict__ X, int64_t npts,
                                                 double *__restrict__ u_out, double *__restrict__ part) {
    constexpr int kMaxCover = 8;   // covering subdomains per dimension (overlap ratio < 7)
    const InstRec &I = insts[s];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ double red[8][4];
    double e2 = 0.0, u2 = 0.0, e1 = 0.0, u1 = 0.0;
    const int d = I.dim;
    // per dimension: centre spacing, half-width and its inverse (the same
    // formulas as the decomposition; the windows vanish on their boundary, so
    // the cover decision there does not change u)
    double sp[3] = {1, 1, 1}, isp[3] = {1, 1, 1}, sg[3] = {1, 1, 1}, isg[3] = {1, 1, 1};
    for (int i = 0; i < d; ++i) {
        double mu0;
        sub_geom(I.lo[i], I.hi[i], I.S[i], I.delta, 0, &mu0, &sg[i]);
        sp[i] = (I.hi[i] - I.lo[i]) / (double)(I.S[i] - 1);
        isp[i] = 1.0 / sp[i];
        isg[i] = 1.0 / sg[i];
    }
    const int H = (int)ceil(I.delta) + 1;
    for (int64_t p = (int64_t)blockIdx.x * 8 + warp; p < npts; p += (int64_t)gridDim.x * 8) {
        double x[3] = {X[3 * p], X[3 * p + 1], X[3 * p + 2]};
        // covering subdomains per dimension: index, local coordinate, window
        // hat (1 + cos(pi s))^2 normalised by the sum over the dimension
        int cj[3][kMaxCover], jn[3] = {1, 1, 1};
        double cs[3][kMaxCover], cw[3][kMaxCover];
        cj[1][0] = cj[2][0] = 0;
        cs[1][0] = cs[2][0] = 0.0;
        cw[1][0] = cw[2][0] = 1.0;
        for (int i = 0; i < d; ++i) {
            const int c = (int)floor((x[i] - I.lo[i]) * isp[i] + 0.5);
            const int a0 = c - H < 0 ? 0 : c - H, a1 = c + H > I.S[i] - 1 ? I.S[i] - 1 : c + H;
            int cnt = 0;
            double W = 0.0;
            for (int l = a0; l <= a1; ++l) {
                const double dx = x[i] - fma(sp[i], (double)l, I.lo[i]);
                if (fabs(dx) < sg[i] && cnt < kMaxCover) {
                    const double sl = dx * isg[i];
                    const double h = 1.0 + cospi(sl);
                    cj[i][cnt] = l;
                    cs[i][cnt] = sl;
                    cw[i][cnt] = h * h;
                    W += h * h;
                    ++cnt;
                }
            }
            const double iW = W > 0.0 ? 1.0 / W : 0.0;
            for (int k = 0; k < cnt; ++k) cw[i][k] *= iW;
            jn[i] = cnt;
        }
        double uh = 0.0;
        const int ncomb = jn[0] * jn[1] * jn[2];
        for (int cmb = 0; cmb < ncomb; ++cmb) {
            int q = cmb;
            int64_t j = 0, stride = 1;
            double w = 1.0;
            float2 tl[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            for (int i = 0; i < d; ++i) {
                const int k = q % jn[i];
                q /= jn[i];
                j += cj[i][k] * stride;
                stride *= I.S[i];
                w *= cw[i][k];
                tl[i] = df_from_double(cs[i][k]);
            }
            const float2 *prm = prm_df + I.prm_off + j * I.K * (d + 1);
            const float2 *aj = a_df + I.col0 + j * I.K;
            float sh = 0.f, sl = 0.f;
            for (int k = lane; k < I.K; k += 32) {
                const float2 *pk = prm + (int64_t)k * (d + 1);
                float2 z = pk[d];
                for (int i = 0; i < d; ++i) z = df_add(z, df_mul(pk[i], tl[i]));
                df_acc(aj[k], df_tanh(z), sh, sl);
            }
            float2 sj2 = make_float2(sh, sl);
            for (int o = 16; o; o >>= 1) sj2 = df_xor_add(sj2, o);
            uh = fma(w, df_to_double(sj2), uh);
        }
        if (lane == 0) {
            u_out[p] = uh;
            const double ue = fam_exact(I, x);
            const double df = uh - ue;
            e2 += df * df;
            u2 += ue * ue;
            e1 += fabs(df);
            u1 += ue;
        }
    }
    if (lane == 0) {
        red[warp][0] = e2; red[warp][1] = u2; red[warp][2] = e1; red[warp][3] = u1;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w][threadIdx.x];
        part[((int64_t)s * kEvalCtas + blockIdx.x) * 4 + threadIdx.x] = t;
    }
}

__global__ void k_eval_finish(const double *__restrict__ part, int s, int nctas, double *__restrict__ err) {
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int c = 0; c < nctas; ++c) t += part[((int64_t)s * kEvalCtas + c) * 4 + threadIdx.x];
        err[4 * s + threadIdx.x] = t;
    }
}

rfm_status launch_eval(const HostPlan &P, void *ws, const double *params, const double *a, const double *X,
                       const int64_t *pt_off, double *u, double *err, cudaStream_t st) {
    const Layout &L = P.L;
    const InstRec *dI = ws_ptr<InstRec>(ws, L.off_inst);
    double *part = ws_ptr<double>(ws, L.off_evpart);
    float2 *evdf = ws_ptr<float2>(ws, L.off_evdf);
    const int64_t n_prm = L.n_prm;
    {
        ProfScope ps("k_eval_split", st);
        const int64_t n = n_prm + L.n_cols;
        const unsigned g = (unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
        k_eval_split<<<g > 0 ? g : 1, 256, 0, st>>>(params, n_prm, a, L.n_cols, evdf);
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    for (int s = 0; s < L.n_inst; ++s) {
        const int64_t n = pt_off[s + 1] - pt_off[s];
        if (n < 0) {
            set_error("rfm_eval: point offsets must be non-decreasing");
            return RFM_EINVAL;
        }
        int g = (int)((n + 7) / 8);
        g = g < 1 ? 1 : (g > kEvalCtas ? kEvalCtas : g);
        const InstRec &I = P.inst[s];
        if (I.depth == 1 && I.act == RFM_ACT_TANH && I.hard_bc == 0.0) {
            ProfScope ps("k_eval", st);
            k_eval_df<<<g, 256, 0, st>>>(dI, s, evdf, evdf + n_prm, X + 3 * pt_off[s], n, u + pt_off[s], part);
        } else {
            // other networks and the hard-constraint ansatz: the FP64 kernel
            ProfScope ps("k_eval", st);
            k_eval<<<g, 256, 0, st>>>(dI, s, params, a, X + 3 * pt_off[s], n, u + pt_off[s], part);
        }
        RFM_CUDA_CHECK(cudaGetLastError());
        if (err) {
            ProfScope ps("k_eval_finish", st);
            k_eval_finish<<<1, 32, 0, st>>>(part, s, g, err);
            RFM_CUDA_CHECK(cudaGetLastError());
        }
    }
    return RFM_OK;
}

}  // namespace rfm

// ---------------------------------------------------------------------------
// Allocation-free evaluation (rfm_eval_noalloc).  Some callers cannot call
// cudaMalloc or own a workspace: code running inside another library's
// memory pool with no allocator hooks, plugin hosts that only hand out input
// and output buffers, or processes whose device memory is fully reserved up
// front.  For them the instance records and the error partials of the
// evaluation live in a fixed static device array instead of a workspace.
// Every GPU that loads the library holds this array until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

namespace rfm {

constexpr int kNoallocMaxInst = 16;   // instances per call
struct NoallocScratch {
    InstRec inst[kNoallocMaxInst];
    double part[kNoallocMaxInst * kEvalCtas * 4];
};
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

// Device address of the scratch array, looked up once per device with that
// device current (in host code the array's name is only a host-side stand-in).
static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[64] = {nullptr};

static rfm_status noalloc_scratch(NoallocScratch **out) {
    int dev = 0;
    RFM_CUDA_CHECK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("rfm_eval_noalloc: device %d out of range", dev);
        return RFM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("rfm_eval_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return RFM_ECUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = reinterpret_cast<NoallocScratch *>(g_noalloc_ptr[dev]);
    return RFM_OK;
}

// One instance record, passed by value (as a kernel parameter), into device
// memory: unlike a copy from host memory that the plan frees on return, a
// parameter is recorded with the launch, so the call can be captured into a
// CUDA graph and replayed.
__global__ void k_put_rec(InstRec *__restrict__ dst, const InstRec rec) {
    const uint64_t *s = reinterpret_cast<const uint64_t *>(&rec);
    uint64_t *d = reinterpret_cast<uint64_t *>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(InstRec) / 8); i += blockDim.x) d[i] = s[i];
}
static_assert(sizeof(InstRec) % 8 == 0 && sizeof(InstRec) <= 4000, "InstRec travels as one kernel parameter");

rfm_status launch_eval_noalloc(const HostPlan &P, const double *params, const double *a, const double *X,
                               const int64_t *pt_off, double *u, double *err, cudaStream_t st) {
    const Layout &L = P.L;
    if (L.n_inst > kNoallocMaxInst) {
        set_error("rfm_eval_noalloc: %d instances exceed its static scratch (at most %d)", L.n_inst,
                  kNoallocMaxInst);
        return RFM_EINVAL;
    }
    NoallocScratch *S = nullptr;
    rfm_status rc = noalloc_scratch(&S);
    if (rc != RFM_OK) return rc;
    for (int s = 0; s < L.n_inst; ++s) {
        k_put_rec<<<1, 32, 0, st>>>(S->inst + s, P.inst[s]);
        RFM_CUDA_CHECK(cudaGetLastError());
    }
    for (int s = 0; s < L.n_inst; ++s) {
        const int64_t n = pt_off[s + 1] - pt_off[s];
        if (n < 0) {
            set_error("rfm_eval_noalloc: point offsets must be non-decreasing");
            return RFM_EINVAL;
        }
        int g = (int)((n + 7) / 8);
        g = g < 1 ? 1 : (g > kEvalCtas ? kEvalCtas : g);
        k_eval<<<g, 256, 0, st>>>(S->inst, s, params, a, X + 3 * pt_off[s], n, u + pt_off[s], S->part);
        RFM_CUDA_CHECK(cudaGetLastError());
        if (err) {
            k_eval_finish<<<1, 32, 0, st>>>(S->part, s, g, err);
            RFM_CUDA_CHECK(cudaGetLastError());
        }
    }
    return RFM_OK;
}

}  // namespace rfm
