// device.cuh -- device functions for points, windows, features and data.
#pragma once
#include "common.cuh"

namespace rfm {

// Row -> point.  Block-local row lr of block B: interior rows first (the
// block's grid box, dimension 0 fastest), then the rows of every face the
// block touches, in face order, each over the block's box in the tangent
// dimensions.  Returns the instance-local global row index; fills x, the
// boundary set (-1 interior), and per dimension the index used in the cover
// tables (grid index, or n+side for the normal dimension of a face).
__device__ inline int64_t block_row_point(const InstRec &I, const BlkRec &B, int lr, double *x, int *kind,
                                          int *gcov) {
    x[0] = x[1] = x[2] = 0.0;
    gcov[0] = gcov[1] = gcov[2] = 0;
    if (lr < B.n_int) {
        int l = lr;
        int64_t r = 0, stride = 1;
        for (int i = 0; i < I.dim; ++i) {
            int g = B.box_lo[i] + l % B.box_n[i];
            l /= B.box_n[i];
            x[i] = grid_coord(I.lo[i], I.hi[i], I.n[i], g);
            gcov[i] = g;
            r += g * stride;
            stride *= I.n[i];
        }
        *kind = -1;
        return r;
    }
    int f = -1;
    for (int ff = 0; ff < I.nfaces; ++ff)
        if (B.face_off[ff] >= 0 && B.face_off[ff] <= lr) f = ff;
    int nd, side;
    face_dims(I.pde, f, &nd, &side);
    int l = lr - B.face_off[f];
    int64_t r = I.face_row0[f], stride = 1;
    for (int i = 0; i < I.dim; ++i) {
        if (i == nd) {
            x[i] = side ? I.hi[i] : I.lo[i];
            gcov[i] = I.n[i] + side;
        } else {
            int g = B.box_lo[i] + l % B.box_n[i];
            l /= B.box_n[i];
            x[i] = grid_coord(I.lo[i], I.hi[i], I.n[i], g);
            gcov[i] = g;
            r += g * stride;
            stride *= I.n[i];
        }
    }
    *kind = face_set_of(I.pde, I.dim, f);
    return r;
}

// Instance-local row r -> point and boundary set (interior grid, then faces).
__device__ inline void row_point(const InstRec &I, int64_t r, double *x, int *kind) {
    x[0] = x[1] = x[2] = 0.0;
    if (r < I.NI) {
        int64_t q = r;
        for (int i = 0; i < I.dim; ++i) {
            int64_t g = q % I.n[i];
            q /= I.n[i];
            x[i] = grid_coord(I.lo[i], I.hi[i], I.n[i], g);
        }
        *kind = -1;
        return;
    }
    int f = 0;
    for (int ff = 0; ff < I.nfaces; ++ff)
        if (I.face_row0[ff] <= r) f = ff;
    int64_t q = r - I.face_row0[f];
    int nd, side;
    face_dims(I.pde, f, &nd, &side);
    for (int i = 0; i < I.dim; ++i) {
        if (i == nd) {
            x[i] = side ? I.hi[i] : I.lo[i];
        } else {
            int64_t g = q % I.n[i];
            q /= I.n[i];
            x[i] = grid_coord(I.lo[i], I.hi[i], I.n[i], g);
        }
    }
    *kind = face_set_of(I.pde, I.dim, f);
}

// One-dimensional normalised window along dimension i for subdomain ji at
// coordinate x, with first and second derivative.  On a tensor-product
// decomposition the sum of the window hats factorises over dimensions, so the
// normalised d-dimensional window is the product of these factors.
__device__ inline void window_1d(const InstRec &I, int i, int ji, double x, double *nu, double *nu1, double *nu2) {
    const int S = I.S[i];
    const int H = (int)ceil(I.delta) + 1;
    double W = 0.0, W1 = 0.0, W2 = 0.0, g = 0.0, g1 = 0.0, g2 = 0.0;
    int lo_j = ji - H < 0 ? 0 : ji - H, hi_j = ji + H > S - 1 ? S - 1 : ji + H;
    for (int l = lo_j; l <= hi_j; ++l) {
        double mu, sig;
        sub_geom(I.lo[i], I.hi[i], S, I.delta, l, &mu, &sig);
        double d = x - mu;
        if (!(fabs(d) < sig)) continue;
        double s = d / sig, sn, c;
        sincospi(s, &sn, &c);
        double a = 1.0 + c;
        double h0 = a * a;
        double h1 = -2.0 * a * sn * (M_PI / sig);
        double h2 = 2.0 * (sn * sn - a * c) * (M_PI * M_PI / (sig * sig));
        W += h0;
        W1 += h1;
        W2 += h2;
        if (l == ji) { g = h0; g1 = h1; g2 = h2; }
    }
    if (W == 0.0 || g == 0.0 && g1 == 0.0 && g2 == 0.0) {
        *nu = *nu1 = *nu2 = 0.0;
        return;
    }
    double iW = 1.0 / W;
    *nu = g * iW;
    *nu1 = g1 * iW - g * W1 * iW * iW;
    *nu2 = g2 * iW - 2.0 * g1 * W1 * iW * iW - g * W2 * iW * iW + 2.0 * g * W1 * W1 * iW * iW * iW;
}

// Normalised window of block B at x with gradient and pure second partials.
__device__ inline void window_nd(const InstRec &I, const int *jd, const double *x, double *w, double *dw, double *d2w) {
    double nu[3], n1[3], n2[3];
    for (int i = 0; i < 3; ++i) { nu[i] = 1.0; n1[i] = 0.0; n2[i] = 0.0; }
    for (int i = 0; i < I.dim; ++i) window_1d(I, i, jd[i], x[i], &nu[i], &n1[i], &n2[i]);
    if (I.hard_bc > 0.0) {
        // hard-constraint ansatz (Sec. 4.1): every factor times
        // g_i = tanh(c (x_i - lo_i)) tanh(c (hi_i - x_i)), by the product rule
        const double c = I.hard_bc;
        for (int i = 0; i < I.dim; ++i) {
            const double A = tanh(c * (x[i] - I.lo[i])), Bt = tanh(c * (I.hi[i] - x[i]));
            const double A1 = c * (1.0 - A * A), B1 = -c * (1.0 - Bt * Bt);
            const double A2 = -2.0 * c * c * A * (1.0 - A * A), B2 = -2.0 * c * c * Bt * (1.0 - Bt * Bt);
            const double g = A * Bt, g1 = A1 * Bt + A * B1, g2 = A2 * Bt + 2.0 * A1 * B1 + A * B2;
            const double v = nu[i], v1 = n1[i], v2 = n2[i];
            nu[i] = g * v;
            n1[i] = g1 * v + g * v1;
            n2[i] = g2 * v + 2.0 * g1 * v1 + g * v2;
        }
    }
    *w = nu[0] * nu[1] * nu[2];
    for (int i = 0; i < 3; ++i) {
        double o = 1.0;
        for (int k = 0; k < 3; ++k)
            if (k != i) o *= nu[k];
        dw[i] = n1[i] * o;
        d2w[i] = n2[i] * o;
    }
}

// Row coefficients: every entry of the row is
//   c0 phi + sum_i c1_i dphi/dx_i + sum_i c2_i d2phi/dx_i^2
// for the row's operator applied to w_j phi (product rule), already scaled by
// the row weight of Eq. (5).  Interior Poisson: -Laplace; interior heat:
// d/dt - kappa Laplace_x; boundary: the trace.
__device__ inline void row_coefficients(const InstRec &I, int kind, double w, const double *dw, const double *d2w,
                                        double *c0, double *c1, double *c2) {
    for (int i = 0; i < 3; ++i) { c1[i] = 0.0; c2[i] = 0.0; }
    if (kind >= 0) {
        if (I.pde == RFM_PDE_OSC && kind == 1) {
            // the oscillator's second initial row: d/dt (w phi)
            *c0 = I.scale_set[1] * dw[0];
            c1[0] = I.scale_set[1] * w;
            return;
        }
        *c0 = I.scale_set[kind] * w;
        return;
    }
    const double sc = I.scale_int;
    if (I.pde == RFM_PDE_OSC) {
        // m (w phi)'' + mu (w phi)' + k w phi
        const double m = I.fam[0], mu = I.fam[1], k = I.fam[2];
        *c0 = sc * (m * d2w[0] + mu * dw[0] + k * w);
        c1[0] = sc * (2.0 * m * dw[0] + mu * w);
        c2[0] = sc * m * w;
        return;
    }
    if (I.pde == RFM_PDE_POISSON) {
        double s2 = 0.0;
        for (int i = 0; i < I.dim; ++i) {
            s2 += d2w[i];
            c1[i] = -2.0 * sc * dw[i];
            c2[i] = -sc * w;
        }
        *c0 = -sc * s2;
    } else {
        const int T = I.dim - 1;
        double s2 = 0.0;
        for (int i = 0; i < T; ++i) {
            s2 += d2w[i];
            c1[i] = -2.0 * I.kappa * sc * dw[i];
            c2[i] = -I.kappa * sc * w;
        }
        *c0 = sc * (dw[T] - I.kappa * s2);
        c1[T] = sc * w;
    }
}

// Closed-form data of the manufactured families.
__device__ inline double fam_exact(const InstRec &I, const double *x) {
    double u = 0.0;
    if (I.family == RFM_FAM_SINPROD) {
        for (int m = 0; m < I.n_modes; ++m) {
            double t = I.fam[4 * m];
            for (int i = 0; i < I.dim; ++i) t *= sinpi(I.fam[4 * m + 1 + i] * x[i]);
            u += t;
        }
        return u;
    }
    if (I.family == RFM_FAM_HEAT_SINPROD) {
        const int T = I.dim - 1;
        for (int m = 0; m < I.n_modes; ++m) {
            double k2 = 0.0, t = I.fam[4 * m];
            for (int i = 0; i < T; ++i) {
                double k = I.fam[4 * m + 1 + i];
                k2 += k * k;
                t *= sinpi(k * x[i]);
            }
            u += t * exp(-I.kappa * M_PI * M_PI * k2 * x[T]);
        }
        return u;
    }
    if (I.family == RFM_FAM_OSC) {
        const double m = I.fam[0], mu = I.fam[1], k = I.fam[2];
        const double d = mu / (2.0 * m), w = sqrt(k / m - d * d), t = x[0] - I.lo[0];
        return exp(-d * t) * (cos(w * t) + d / w * sin(w * t));
    }
    return __longlong_as_double(0x7ff8000000000000ULL);
}

__device__ inline double fam_source(const InstRec &I, const double *x) {
    if (I.family == RFM_FAM_SINPROD) {
        double f = 0.0;
        for (int m = 0; m < I.n_modes; ++m) {
            double k2 = 0.0, t = I.fam[4 * m];
            for (int i = 0; i < I.dim; ++i) {
                double k = I.fam[4 * m + 1 + i];
                k2 += k * k;
                t *= sinpi(k * x[i]);
            }
            f += t * (M_PI * M_PI) * k2;
        }
        return f;
    }
    if (I.family == RFM_FAM_HEAT_SINPROD || I.family == RFM_FAM_OSC) return 0.0;
    const double *p = I.fam;
    return sinpi(p[0] * x[0]) * sinpi(p[1] * x[1]) + p[2] * sinpi(p[3] * x[0] + p[4] * x[1]);
}

// Data of boundary set `kind` (the oscillator's set 1 is u'(lo)).
__device__ inline double fam_bdata(const InstRec &I, const double *x, int kind) {
    if (I.family == RFM_FAM_OSC && kind == 1) {
        const double m = I.fam[0], mu = I.fam[1], k = I.fam[2];
        const double d = mu / (2.0 * m), w = sqrt(k / m - d * d), t = x[0] - I.lo[0];
        return -(d * d / w + w) * exp(-d * t) * sin(w * t);
    }
    return I.family == RFM_FAM_PARAM5 ? 0.0 : fam_exact(I, x);
}

// Activation Xi of the subdomain networks and its first two derivatives.
__device__ inline void act_eval(int act, double s, double *f, double *f1, double *f2) {
    if (act == RFM_ACT_SIGMOID) {
        const double g = 1.0 / (1.0 + exp(-s));
        *f = g;
        *f1 = g * (1.0 - g);
        *f2 = g * (1.0 - g) * (1.0 - 2.0 * g);
    } else if (act == RFM_ACT_SIN) {
        double sn, cs;
        sincos(s, &sn, &cs);
        *f = sn;
        *f1 = cs;
        *f2 = -sn;
    } else {
        const double t = tanh(s);
        *f = t;
        *f1 = 1.0 - t * t;
        *f2 = -2.0 * t * (1.0 - t * t);
    }
}
__device__ inline void act_eval(int act, float s, float *f, float *f1, float *f2) {
    if (act == RFM_ACT_SIGMOID) {
        const float g = 1.f / (1.f + expf(-s));
        *f = g;
        *f1 = g * (1.f - g);
        *f2 = g * (1.f - g) * (1.f - 2.f * g);
    } else if (act == RFM_ACT_SIN) {
        float sn, cs;
        sincosf(s, &sn, &cs);
        *f = sn;
        *f1 = cs;
        *f2 = -sn;
    } else {
        const float t = tanhf(s);
        *f = t;
        *f1 = 1.f - t * t;
        *f2 = -2.f * t * (1.f - t * t);
    }
}

// Output-layer input z of subdomain network `prm_j` (Eq. (2) with h - 1
// hidden layers of K units) at the normalised point xn = (x - mu)/sig, with
// (when dz is not null) its partial derivatives dz[i * kMaxDeepK + m] and pure
// second partials d2z[...] with respect to x_i (forward propagation; the
// input's derivatives are 1/sig_i).  Writes I.n_last entries (the point
// itself when h = 1); with hidden layers K <= kMaxDeepK.
__device__ inline void net_hidden(const InstRec &I, const double *prm_j, const double *xn, const double *isg,
                                  double *z, double *dz, double *d2z) {
    const int d = I.dim, K = I.K;
    double a[kMaxDeepK], da[3][kMaxDeepK], d2a[3][kMaxDeepK];
    int nin = d;
    for (int m = 0; m < d; ++m) {
        a[m] = xn[m];
        for (int i = 0; i < 3; ++i) {
            da[i][m] = i == m ? isg[m] : 0.0;
            d2a[i][m] = 0.0;
        }
    }
    const double *q = prm_j + (int64_t)K * (I.n_last + 1);
    for (int l = 1; l < I.depth; ++l) {
        double na[kMaxDeepK], nda[3][kMaxDeepK], nd2a[3][kMaxDeepK];
        const double *W = q, *b = q + (int64_t)K * nin;
        for (int u = 0; u < K; ++u) {
            double p = b[u], dp[3] = {0, 0, 0}, d2p[3] = {0, 0, 0};
            for (int m = 0; m < nin; ++m) {
                const double wum = W[u * nin + m];
                p = fma(wum, a[m], p);
                if (dz)
                    for (int i = 0; i < d; ++i) {
                        dp[i] = fma(wum, da[i][m], dp[i]);
                        d2p[i] = fma(wum, d2a[i][m], d2p[i]);
                    }
            }
            double f, f1, f2;
            act_eval(I.act, p, &f, &f1, &f2);
            na[u] = f;
            for (int i = 0; i < d; ++i) {
                nda[i][u] = f1 * dp[i];
                nd2a[i][u] = f2 * dp[i] * dp[i] + f1 * d2p[i];
            }
        }
        q += (int64_t)K * (nin + 1);
        nin = K;
        for (int u = 0; u < K; ++u) {
            a[u] = na[u];
            for (int i = 0; i < d; ++i) {
                da[i][u] = nda[i][u];
                d2a[i][u] = nd2a[i][u];
            }
        }
    }
    for (int u = 0; u < nin; ++u) {
        z[u] = a[u];
        if (dz)
            for (int i = 0; i < 3; ++i) {
                dz[i * kMaxDeepK + u] = i < d ? da[i][u] : 0.0;
                d2z[i * kMaxDeepK + u] = i < d ? d2a[i][u] : 0.0;
            }
    }
}

}  // namespace rfm
