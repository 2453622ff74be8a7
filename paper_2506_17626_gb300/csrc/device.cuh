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
    int nd = f / 2, side = f % 2;
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
    *kind = (I.pde == RFM_PDE_HEAT && nd == I.dim - 1) ? 1 : 0;
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
    int nd = f / 2, side = f % 2;
    for (int i = 0; i < I.dim; ++i) {
        if (i == nd) {
            x[i] = side ? I.hi[i] : I.lo[i];
        } else {
            int64_t g = q % I.n[i];
            q /= I.n[i];
            x[i] = grid_coord(I.lo[i], I.hi[i], I.n[i], g);
        }
    }
    *kind = (I.pde == RFM_PDE_HEAT && nd == I.dim - 1) ? 1 : 0;
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
        *c0 = I.scale_set[kind] * w;
        return;
    }
    const double sc = I.scale_int;
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
    if (I.family == RFM_FAM_HEAT_SINPROD) return 0.0;
    const double *p = I.fam;
    return sinpi(p[0] * x[0]) * sinpi(p[1] * x[1]) + p[2] * sinpi(p[3] * x[0] + p[4] * x[1]);
}

__device__ inline double fam_bdata(const InstRec &I, const double *x) {
    return I.family == RFM_FAM_PARAM5 ? 0.0 : fam_exact(I, x);
}

}  // namespace rfm
