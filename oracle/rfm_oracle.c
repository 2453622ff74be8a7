/*
 * rfm_oracle.c -- plain, slow, FP64 CPU oracle for the ELM-FBPINN hot path with
 * local RRQR filtering and right preconditioning (van Beek, Dolean, Moseley,
 * "Local Feature Filtering for Scalable and Well-Conditioned Domain-Decomposed
 * Random Feature Methods").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA library is
 * checked against.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load it; the library never calls it and shares no code with it.
 *
 * Every function writes out a definition from the paper directly, with plain
 * loops and no blocking, fusion or reordering:
 *   - ansatz, features and loss rows: Sec. 2.1, Eqs. (1)-(5) and the entry
 *     formulas for N and B that follow Eq. (5);
 *   - block structure: Eq. (6) (row sets I_j = {r : w_j(x_r) != 0});
 *   - decomposition and windows: Sec. 4.2 (overlapping box decomposition and
 *     the normalised cosine window);
 *   - local filtering: Algorithm 1 with the threshold taken relative to the
 *     leading diagonal entry of R_j (Sec. 3.1), computed by Householder QR
 *     with column pivoting (Businger-Golub), column norms recomputed exactly at
 *     every step;
 *   - preconditioner: Sec. 3.2 (S^-1 = sum_j W_j^T R_j^-1 W_j by substitution)
 *     and Proposition 3.1 (explicit Q_j, used only as a check);
 *   - solver: Algorithm 2 with LSQR (Paige and Saunders 1982), output a with
 *     zeros at dropped columns.
 * Where the paper is silent, ambiguous or garbled, the reading taken is stated
 * at the function whose arithmetic it decides.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { PDE_POISSON = 0, PDE_HEAT = 1, PDE_OSC = 2 };
enum { FAM_SINPROD = 0, FAM_HEAT_SINPROD = 1, FAM_PARAM5 = 2, FAM_OSC = 3 };
enum { ACT_TANH = 0, ACT_SIGMOID = 1, ACT_SIN = 2 };

/* One problem instance.  depth is h of Eq. (2) (0 is read as 1), act the
 * activation Xi, hard_bc > 0 the factor c of the hard-constraint ansatz of the
 * Laplace problem (Sec. 4.1).  The damped oscillator (PDE_OSC, Sec. 4.1) takes
 * its coefficients m, mu, k from fam[0], fam[1], fam[2]. */
typedef struct {
    int32_t dim, pde, family, n_modes;
    int32_t S[3], n[3];
    int32_t K, pad0;
    double delta, kappa;
    double lo[3], hi[3];
    double lam[2];
    double fam[64];
    int32_t depth, act;
    double hard_bc;
} orc_problem;

/* ------------------------------------------------------------------------ */
/* collocation points: cell-centred interior grid, then boundary faces       */
/* ------------------------------------------------------------------------ */

static int64_t n_interior(const orc_problem *P) {
    int64_t c = 1;
    for (int i = 0; i < P->dim; ++i) c *= P->n[i];
    return c;
}

/* Faces in order: dimension 0 lo, dimension 0 hi, dimension 1 lo, ...  For the
 * heat equation the last coordinate is time and only its lo face (the initial
 * condition) carries data. */
static int n_faces(const orc_problem *P) {
    if (P->hard_bc > 0.0) return 0;   /* the ansatz satisfies the boundary condition: no boundary rows */
    if (P->pde == PDE_OSC) return 2;  /* u(t0) and du/dt(t0): two rows at the initial time */
    return P->pde == PDE_HEAT ? 2 * (P->dim - 1) + 1 : 2 * P->dim;
}

static void face_info(const orc_problem *P, int f, int *normal, int *side) {
    if (P->pde == PDE_OSC) {
        *normal = 0;
        *side = 0;
        return;
    }
    *normal = f / 2;
    *side = f % 2;
}

static int64_t face_points(const orc_problem *P, int f) {
    int nd, sd;
    face_info(P, f, &nd, &sd);
    int64_t c = 1;
    for (int i = 0; i < P->dim; ++i)
        if (i != nd) c *= P->n[i];
    return c;
}

/* boundary set of a face: Poisson has one Dirichlet set; heat has the lateral
 * Dirichlet set (0) and the initial-condition set (1). */
static int face_set(const orc_problem *P, int f) {
    int nd, sd;
    face_info(P, f, &nd, &sd);
    if (P->pde == PDE_OSC) return f;   /* 0: value, 1: first derivative */
    if (P->pde == PDE_HEAT && nd == P->dim - 1) return 1;
    return 0;
}

int64_t orc_num_interior(const orc_problem *P) { return n_interior(P); }

int64_t orc_num_boundary(const orc_problem *P) {
    int64_t c = 0;
    for (int f = 0; f < n_faces(P); ++f) c += face_points(P, f);
    return c;
}

int64_t orc_num_set(const orc_problem *P, int l) {
    int64_t c = 0;
    for (int f = 0; f < n_faces(P); ++f)
        if (face_set(P, f) == l) c += face_points(P, f);
    return c;
}

static double grid_coord(const orc_problem *P, int i, int64_t g) {
    return P->lo[i] + ((double)g + 0.5) * (P->hi[i] - P->lo[i]) / (double)P->n[i];
}

/* Coordinates of global row r.  kind = -1 for an interior row, else the
 * boundary set index. */
void orc_row_point(const orc_problem *P, int64_t r, double *x, int *kind) {
    int64_t NI = n_interior(P);
    x[0] = x[1] = x[2] = 0.0;
    if (r < NI) {
        int64_t q = r;
        for (int i = 0; i < P->dim; ++i) {
            int64_t g = q % P->n[i];
            q /= P->n[i];
            x[i] = grid_coord(P, i, g);
        }
        *kind = -1;
        return;
    }
    int64_t q = r - NI;
    for (int f = 0; f < n_faces(P); ++f) {
        int64_t c = face_points(P, f);
        if (q < c) {
            int nd, sd;
            face_info(P, f, &nd, &sd);
            for (int i = 0; i < P->dim; ++i) {
                if (i == nd) {
                    x[i] = sd ? P->hi[i] : P->lo[i];
                } else {
                    int64_t g = q % P->n[i];
                    q /= P->n[i];
                    x[i] = grid_coord(P, i, g);
                }
            }
            *kind = face_set(P, f);
            return;
        }
        q -= c;
    }
    *kind = -2; /* out of range */
}

/* ------------------------------------------------------------------------ */
/* decomposition and windows (Sec. 4.2)                                      */
/* ------------------------------------------------------------------------ */

/* Subdomain j (lexicographic, dimension 0 fastest).  Centre and half-width per
 * dimension from the overlapping box formula: the box along dimension i is
 * [a + (b-a)((j_i-1) - delta/2)/(S-1), a + (b-a)((j_i-1) + delta/2)/(S-1)]
 * with 1-based j_i, i.e. centre a + (b-a) j_i/(S-1) for 0-based j_i and
 * half-width (b-a) delta / (2 (S-1)). */
void orc_subdomain(const orc_problem *P, int64_t j, double *mu, double *sig) {
    int64_t q = j;
    for (int i = 0; i < 3; ++i) { mu[i] = 0.0; sig[i] = 1.0; }
    for (int i = 0; i < P->dim; ++i) {
        int64_t ji = q % P->S[i];
        q /= P->S[i];
        double L = P->hi[i] - P->lo[i];
        mu[i] = P->lo[i] + L * (double)ji / (double)(P->S[i] - 1);
        sig[i] = L * P->delta / (2.0 * (double)(P->S[i] - 1));
    }
}

int64_t orc_num_subdomains(const orc_problem *P) {
    int64_t c = 1;
    for (int i = 0; i < P->dim; ++i) c *= P->S[i];
    return c;
}

/* Unnormalised window hat_w_j(x) = prod_i [1 + cos(pi (x_i - mu_i)/sig_i)]^2
 * inside the open box |x_i - mu_i| < sig_i and 0 outside, with its first and
 * pure second partial derivatives in every dimension. */
double orc_window_hat(const orc_problem *P, int64_t j, const double *x, double *dw, double *d2w) {
    double mu[3], sig[3];
    orc_subdomain(P, j, mu, sig);
    double g[3], g1[3], g2[3];
    for (int i = 0; i < P->dim; ++i) {
        double s = (x[i] - mu[i]) / sig[i];
        if (!(fabs(x[i] - mu[i]) < sig[i])) {
            for (int k = 0; k < P->dim; ++k) { dw[k] = 0.0; d2w[k] = 0.0; }
            return 0.0;
        }
        double c = cos(M_PI * s), sn = sin(M_PI * s);
        g[i] = (1.0 + c) * (1.0 + c);
        g1[i] = -2.0 * (1.0 + c) * sn * M_PI / sig[i];
        g2[i] = 2.0 * (sn * sn - (1.0 + c) * c) * M_PI * M_PI / (sig[i] * sig[i]);
    }
    double w = 1.0;
    for (int i = 0; i < P->dim; ++i) w *= g[i];
    for (int i = 0; i < P->dim; ++i) {
        double o = 1.0;
        for (int k = 0; k < P->dim; ++k)
            if (k != i) o *= g[k];
        dw[i] = g1[i] * o;
        d2w[i] = g2[i] * o;
    }
    return w;
}

/* Normalised window w_j = hat_w_j / sum_l hat_w_l (partition of unity), and
 * its partial derivatives by the quotient rule. */
double orc_window(const orc_problem *P, int64_t j, const double *x, double *dw, double *d2w) {
    double hd[3] = {0, 0, 0}, hd2[3] = {0, 0, 0};
    double h = orc_window_hat(P, j, x, hd, hd2);
    double W = 0.0, Wd[3] = {0, 0, 0}, Wd2[3] = {0, 0, 0};
    int64_t J = orc_num_subdomains(P);
    for (int64_t l = 0; l < J; ++l) {
        double ld[3] = {0, 0, 0}, ld2[3] = {0, 0, 0};
        double hl = orc_window_hat(P, l, x, ld, ld2);
        W += hl;
        for (int i = 0; i < P->dim; ++i) { Wd[i] += ld[i]; Wd2[i] += ld2[i]; }
    }
    for (int i = 0; i < 3; ++i) { dw[i] = 0.0; d2w[i] = 0.0; }
    if (W == 0.0) return 0.0;
    for (int i = 0; i < P->dim; ++i) {
        dw[i] = hd[i] / W - h * Wd[i] / (W * W);
        d2w[i] = hd2[i] / W - 2.0 * hd[i] * Wd[i] / (W * W) - h * Wd2[i] / (W * W)
               + 2.0 * h * Wd[i] * Wd[i] / (W * W * W);
    }
    return h / W;
}

/* ------------------------------------------------------------------------ */
/* data of the manufactured problems                                         */
/* ------------------------------------------------------------------------ */

/* exact solution (NaN when the family has no closed form) */
double orc_exact(const orc_problem *P, const double *x) {
    double u = 0.0;
    if (P->family == FAM_SINPROD) {
        for (int m = 0; m < P->n_modes; ++m) {
            double t = P->fam[4 * m];
            for (int i = 0; i < P->dim; ++i) t *= sin(P->fam[4 * m + 1 + i] * M_PI * x[i]);
            u += t;
        }
        return u;
    }
    if (P->family == FAM_HEAT_SINPROD) {
        int ds = P->dim - 1;
        for (int m = 0; m < P->n_modes; ++m) {
            double k2 = 0.0, t = P->fam[4 * m];
            for (int i = 0; i < ds; ++i) {
                double k = P->fam[4 * m + 1 + i];
                k2 += k * k;
                t *= sin(k * M_PI * x[i]);
            }
            u += t * exp(-P->kappa * M_PI * M_PI * k2 * x[ds]);
        }
        return u;
    }
    if (P->family == FAM_OSC) {
        /* under-damped oscillator m u'' + mu u' + k u = 0 with u(t0) = 1,
         * u'(t0) = 0: u = e^{-d s}(cos(w s) + (d/w) sin(w s)), s = t - t0,
         * d = mu/(2m), w = sqrt(k/m - d^2) (Sec. 4.1) */
        double m = P->fam[0], mu = P->fam[1], k = P->fam[2];
        double d = mu / (2.0 * m), w = sqrt(k / m - d * d), t = x[0] - P->lo[0];
        return exp(-d * t) * (cos(w * t) + d / w * sin(w * t));
    }
    return NAN;
}

/* du/dt of the oscillator's exact solution (the data of its derivative row) */
static double osc_exact_dt(const orc_problem *P, const double *x) {
    double m = P->fam[0], mu = P->fam[1], k = P->fam[2];
    double d = mu / (2.0 * m), w = sqrt(k / m - d * d), t = x[0] - P->lo[0];
    /* d/dt of e^{-dt}(cos wt + (d/w) sin wt) = -(d^2/w + w) e^{-dt} sin wt */
    return -(d * d / w + w) * exp(-d * t) * sin(w * t);
}

/* right-hand side f of the PDE at an interior point */
double orc_source(const orc_problem *P, const double *x) {
    if (P->family == FAM_SINPROD) {
        /* f = -Laplace u */
        double f = 0.0;
        for (int m = 0; m < P->n_modes; ++m) {
            double k2 = 0.0, t = P->fam[4 * m];
            for (int i = 0; i < P->dim; ++i) {
                double k = P->fam[4 * m + 1 + i];
                k2 += k * k;
                t *= sin(k * M_PI * x[i]);
            }
            f += t * M_PI * M_PI * k2;
        }
        return f;
    }
    if (P->family == FAM_HEAT_SINPROD || P->family == FAM_OSC) return 0.0; /* homogeneous equations */
    if (P->family == FAM_PARAM5) {
        const double *p = P->fam;
        return sin(p[0] * M_PI * x[0]) * sin(p[1] * M_PI * x[1])
             + p[2] * sin(p[3] * M_PI * x[0] + p[4] * M_PI * x[1]);
    }
    return NAN;
}

/* boundary / initial data g_l of boundary set `kind` at a boundary point */
static double bdata_set(const orc_problem *P, const double *x, int kind) {
    if (P->family == FAM_PARAM5) return 0.0;
    if (P->pde == PDE_OSC && kind == 1) return osc_exact_dt(P, x);
    return orc_exact(P, x);
}

double orc_bdata(const orc_problem *P, const double *x) { return bdata_set(P, x, 0); }
double orc_bdata_set(const orc_problem *P, const double *x, int kind) { return bdata_set(P, x, kind); }

/* ------------------------------------------------------------------------ */
/* assembly (Sec. 2.1, entry formulas after Eq. (5); Eq. (6))                 */
/* ------------------------------------------------------------------------ */

/* Row set I_j = {r : w_j(x_r) != 0} in increasing global row order.  The
 * window is nonzero exactly on the open box |x_i - mu_i| < sig_i, and that
 * test is what decides membership (it does not depend on how cos rounds next
 * to the box edge).  Returns |I_j|; fills grow when non-NULL. */
int64_t orc_block_rows(const orc_problem *P, int64_t j, int64_t *grow) {
    int64_t N = n_interior(P) + orc_num_boundary(P);
    double mu[3], sig[3];
    orc_subdomain(P, j, mu, sig);
    int64_t c = 0;
    for (int64_t r = 0; r < N; ++r) {
        double x[3];
        int kind, inside = 1;
        orc_row_point(P, r, x, &kind);
        for (int i = 0; i < P->dim; ++i)
            if (!(fabs(x[i] - mu[i]) < sig[i])) inside = 0;
        if (inside) {
            if (grow) grow[c] = r;
            ++c;
        }
    }
    return c;
}

/* ---- the subdomain networks of Eq. (2) ---------------------------------- */

static int depth_of(const orc_problem *P) { return P->depth > 1 ? P->depth : 1; }

/* Inputs of the output layer: d for a one-layer network (the normalised
 * coordinates), else K (the last hidden layer's width; hidden layers are K
 * wide). */
static int n_last(const orc_problem *P) { return depth_of(P) > 1 ? P->K : P->dim; }

/* Parameters of one subdomain network, laid out as: the output layer, one row
 * (w_1 .. w_nlast, b) per feature k; then hidden layers l = 1 .. h-1, each its
 * weights W^(l) (K x n_{l-1}, row-major) followed by its biases b^(l) (K),
 * with n_0 = dim.  For h = 1 this is (k, [w_1..w_d, b]). */
int64_t orc_params_per_subdomain(const orc_problem *P) {
    int64_t c = (int64_t)P->K * (n_last(P) + 1);
    int nin = P->dim;
    for (int l = 1; l < depth_of(P); ++l) {
        c += (int64_t)P->K * (nin + 1);
        nin = P->K;
    }
    return c;
}

/* Activation Xi and its first two derivatives. */
static void activation(const orc_problem *P, double s, double *f, double *f1, double *f2) {
    if (P->act == ACT_SIGMOID) {
        double g = 1.0 / (1.0 + exp(-s));
        *f = g;
        *f1 = g * (1.0 - g);
        *f2 = g * (1.0 - g) * (1.0 - 2.0 * g);
    } else if (P->act == ACT_SIN) {
        *f = sin(s);
        *f1 = cos(s);
        *f2 = -sin(s);
    } else {
        double t = tanh(s);
        *f = t;
        *f1 = 1.0 - t * t;
        *f2 = -2.0 * t * (1.0 - t * t);
    }
}

#define ORC_MAXH 128   /* widest layer input the oracle handles */

/* Input of the output layer of subdomain j's network at x, with its partial
 * derivatives dz[i][m] = d z_m / d x_i and pure second partials d2z[i][m]
 * (forward propagation of value, gradient and second partials through the
 * hidden layers of Eq. (2); the network input is (x - mu)/sig, the subdomain
 * normalisation of Sec. 4.2).  Returns the input width. */
static int last_hidden(const orc_problem *P, const double *prm_j, const double *mu, const double *sig,
                       const double *x, double *z, double dz[3][ORC_MAXH], double d2z[3][ORC_MAXH]) {
    int nin = P->dim;
    for (int m = 0; m < nin; ++m) {
        z[m] = (x[m] - mu[m]) / sig[m];
        for (int i = 0; i < 3; ++i) {
            dz[i][m] = (i == m) ? 1.0 / sig[m] : 0.0;
            d2z[i][m] = 0.0;
        }
    }
    const double *q = prm_j + (int64_t)P->K * (n_last(P) + 1);
    for (int l = 1; l < depth_of(P); ++l) {
        double nz[ORC_MAXH], ndz[3][ORC_MAXH], nd2z[3][ORC_MAXH];
        const double *W = q, *b = q + (int64_t)P->K * nin;
        for (int u = 0; u < P->K; ++u) {
            double p = b[u], dp[3] = {0, 0, 0}, d2p[3] = {0, 0, 0};
            for (int m = 0; m < nin; ++m) {
                double wum = W[(int64_t)u * nin + m];
                p += wum * z[m];
                for (int i = 0; i < P->dim; ++i) {
                    dp[i] += wum * dz[i][m];
                    d2p[i] += wum * d2z[i][m];
                }
            }
            double f, f1, f2;
            activation(P, p, &f, &f1, &f2);
            nz[u] = f;
            for (int i = 0; i < 3; ++i) {
                ndz[i][u] = i < P->dim ? f1 * dp[i] : 0.0;
                nd2z[i][u] = i < P->dim ? f2 * dp[i] * dp[i] + f1 * d2p[i] : 0.0;
            }
        }
        q += (int64_t)P->K * (nin + 1);
        nin = P->K;
        for (int u = 0; u < nin; ++u) {
            z[u] = nz[u];
            for (int i = 0; i < 3; ++i) {
                dz[i][u] = ndz[i][u];
                d2z[i][u] = nd2z[i][u];
            }
        }
    }
    return nin;
}

/* Feature phi_jk = Xi(w_k . z + b_k) on the output layer's input z (for a
 * one-layer network z = (x - mu)/sig, the normalised coordinates of Sec. 4.2,
 * with a bias), with gradient and pure second partials by the chain rule. */
static void feature_from(const orc_problem *P, const double *prm_k, int nin, const double *z,
                         double dz[3][ORC_MAXH], double d2z[3][ORC_MAXH], double *phi, double *dphi,
                         double *d2phi) {
    double s = prm_k[nin], ds[3] = {0, 0, 0}, d2s[3] = {0, 0, 0};
    for (int m = 0; m < nin; ++m) {
        s += prm_k[m] * z[m];
        for (int i = 0; i < P->dim; ++i) {
            ds[i] += prm_k[m] * dz[i][m];
            d2s[i] += prm_k[m] * d2z[i][m];
        }
    }
    double f, f1, f2;
    activation(P, s, &f, &f1, &f2);
    *phi = f;
    for (int i = 0; i < 3; ++i) {
        dphi[i] = i < P->dim ? f1 * ds[i] : 0.0;
        d2phi[i] = i < P->dim ? f2 * ds[i] * ds[i] + f1 * d2s[i] : 0.0;
    }
}

/* The hard-constraint factor of the Laplace ansatz (Sec. 4.1),
 * g(x) = prod_i tanh(c (x_i - a_i)) tanh(c (b_i - x_i)), with gradient and pure
 * second partials; g = 1 when hard_bc is 0. */
static double hard_factor(const orc_problem *P, const double *x, double *dg, double *d2g) {
    double gi[3], g1[3], g2[3];
    for (int i = 0; i < 3; ++i) { gi[i] = 1.0; g1[i] = 0.0; g2[i] = 0.0; }
    if (P->hard_bc > 0.0) {
        double c = P->hard_bc;
        for (int i = 0; i < P->dim; ++i) {
            double A = tanh(c * (x[i] - P->lo[i])), B = tanh(c * (P->hi[i] - x[i]));
            double A1 = c * (1.0 - A * A), B1 = -c * (1.0 - B * B);
            double A2 = -2.0 * c * c * A * (1.0 - A * A), B2 = -2.0 * c * c * B * (1.0 - B * B);
            gi[i] = A * B;
            g1[i] = A1 * B + A * B1;
            g2[i] = A2 * B + 2.0 * A1 * B1 + A * B2;
        }
    }
    double g = 1.0;
    for (int i = 0; i < P->dim; ++i) g *= gi[i];
    for (int i = 0; i < 3; ++i) {
        double o = 1.0;
        for (int k = 0; k < P->dim; ++k)
            if (k != i) o *= gi[k];
        dg[i] = i < P->dim ? g1[i] * o : 0.0;
        d2g[i] = i < P->dim ? g2[i] * o : 0.0;
    }
    return g;
}

/* The function multiplying each feature of subdomain j: the window w_j, times
 * the hard-constraint factor g when the ansatz has one (product rule). */
static double window_ansatz(const orc_problem *P, int64_t j, const double *x, double *dw, double *d2w) {
    double wd[3] = {0, 0, 0}, wd2[3] = {0, 0, 0}, gd[3], gd2[3];
    double w = orc_window(P, j, x, wd, wd2);
    double g = hard_factor(P, x, gd, gd2);
    for (int i = 0; i < 3; ++i) {
        dw[i] = gd[i] * w + g * wd[i];
        d2w[i] = gd2[i] * w + 2.0 * gd[i] * wd[i] + g * wd2[i];
    }
    return g * w;
}

/* One entry of M for the function v = w phi (w the window, times g with the
 * hard constraint): interior rows carry N[v](x)/sqrt(N_I); boundary rows carry
 * sqrt(lambda_l/N_B^(l)) B_l[v](x), with B_l the trace, or for the
 * oscillator's second initial condition the first derivative. */
static double entry(const orc_problem *P, const double *x, int kind, double w, const double *dw,
                    const double *d2w, double phi, const double *dphi, const double *d2phi) {
    if (kind >= 0) {
        double NB = (double)orc_num_set(P, kind);
        double b = w * phi;
        if (P->pde == PDE_OSC && kind == 1) b = dw[0] * phi + w * dphi[0];
        return sqrt(P->lam[kind] / NB) * b;
    }
    double NI = (double)n_interior(P);
    if (P->pde == PDE_OSC) {
        /* m v'' + mu v' + k v */
        double v0 = w * phi;
        double v1 = dw[0] * phi + w * dphi[0];
        double v2 = d2w[0] * phi + 2.0 * dw[0] * dphi[0] + w * d2phi[0];
        return (P->fam[0] * v2 + P->fam[1] * v1 + P->fam[2] * v0) / sqrt(NI);
    }
    double lap = 0.0;
    int nsp = P->pde == PDE_HEAT ? P->dim - 1 : P->dim;
    for (int i = 0; i < nsp; ++i)
        lap += d2w[i] * phi + 2.0 * dw[i] * dphi[i] + w * d2phi[i];
    double v;
    if (P->pde == PDE_HEAT) {
        int T = P->dim - 1;
        double dt = dw[T] * phi + w * dphi[T];
        v = dt - P->kappa * lap;
    } else {
        v = -lap;
    }
    return v / sqrt(NI);
}

/* Block M_j = M restricted to I_j x K_j, column-major m x K with ld = m.
 * params holds orc_params_per_subdomain doubles per subdomain, subdomains in
 * order (for one-layer networks (J, K, dim+1) row-major). */
void orc_assemble_block(const orc_problem *P, const double *params, int64_t j, const int64_t *grow,
                        int64_t m, double *Mj) {
    double mu[3], sig[3];
    orc_subdomain(P, j, mu, sig);
    const int64_t np = orc_params_per_subdomain(P);
    const double *pj = params + j * np;
    const int nl = n_last(P);
    for (int64_t lr = 0; lr < m; ++lr) {
        double x[3], dw[3], d2w[3];
        int kind;
        orc_row_point(P, grow[lr], x, &kind);
        double w = window_ansatz(P, j, x, dw, d2w);
        double z[ORC_MAXH], dz[3][ORC_MAXH], d2z[3][ORC_MAXH];
        int nin = last_hidden(P, pj, mu, sig, x, z, dz, d2z);
        for (int k = 0; k < P->K; ++k) {
            double phi, dphi[3], d2phi[3];
            feature_from(P, pj + (int64_t)k * (nl + 1), nin, z, dz, d2z, &phi, dphi, d2phi);
            Mj[(size_t)k * m + lr] = entry(P, x, kind, w, dw, d2w, phi, dphi, d2phi);
        }
    }
}

/* Right-hand side h = [f / sqrt(N_I); sqrt(lambda_l/N_B^(l)) g] over all rows. */
void orc_rhs(const orc_problem *P, double *h) {
    int64_t NI = n_interior(P), N = NI + orc_num_boundary(P);
    for (int64_t r = 0; r < N; ++r) {
        double x[3];
        int kind;
        orc_row_point(P, r, x, &kind);
        if (kind < 0)
            h[r] = orc_source(P, x) / sqrt((double)NI);
        else
            h[r] = sqrt(P->lam[kind] / (double)orc_num_set(P, kind)) * bdata_set(P, x, kind);
    }
}

/* Dense global matrix (N x J K, column-major, ld = N) for small problems,
 * built from the definition entry by entry: M_{r,l} with l = j K + k. */
void orc_assemble_dense(const orc_problem *P, const double *params, double *M) {
    int64_t N = n_interior(P) + orc_num_boundary(P);
    int64_t J = orc_num_subdomains(P);
    const int64_t np = orc_params_per_subdomain(P);
    const int nl = n_last(P);
    for (int64_t j = 0; j < J; ++j) {
        double mu[3], sig[3];
        orc_subdomain(P, j, mu, sig);
        for (int64_t r = 0; r < N; ++r) {
            double x[3], dw[3], d2w[3];
            int kind;
            orc_row_point(P, r, x, &kind);
            double w = window_ansatz(P, j, x, dw, d2w);
            double z[ORC_MAXH], dz[3][ORC_MAXH], d2z[3][ORC_MAXH];
            int nin = last_hidden(P, params + j * np, mu, sig, x, z, dz, d2z);
            for (int k = 0; k < P->K; ++k) {
                double phi, dphi[3], d2phi[3];
                feature_from(P, params + j * np + (int64_t)k * (nl + 1), nin, z, dz, d2z, &phi, dphi, d2phi);
                M[(size_t)(j * P->K + k) * N + r] = entry(P, x, kind, w, dw, d2w, phi, dphi, d2phi);
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* local filtering: sigma-RRQR by QR with column pivoting (Algorithm 1)      */
/* ------------------------------------------------------------------------ */

static double col_norm(const double *a, int64_t len) {
    double s = 0.0;
    for (int64_t i = 0; i < len; ++i) s += a[i] * a[i];
    return sqrt(s);
}

/* Householder QR with column pivoting of the m x n column-major matrix A
 * (leading dimension lda), stopped at the first step k whose pivot norm
 * |R_kk| is zero or below tol * |R_11| (strict; the threshold is relative to
 * the leading diagonal value of R, Sec. 3.1).  On return A holds R in its
 * upper triangle and the Householder vectors (unit first entry implied) below
 * it, tau the reflector scalars, perm[c] the original index of column c.
 * Pivot: the trailing column of largest norm, recomputed exactly at every
 * step; ties go to the lowest original index.  Reflector for x = A[k:m, k]:
 * beta = -sign(x_0) ||x|| (sign(0) = +), v = x / (x_0 - beta) with v_0 = 1,
 * tau = (beta - x_0) / beta, so that (I - tau v v^T) x = beta e_1.
 * Returns the number of kept columns r; *r11 receives |R_11|. */
int orc_qrcp(int m, int n, double *A, int lda, double tol, int *perm, double *tau, double *r11) {
    for (int c = 0; c < n; ++c) perm[c] = c;
    int steps = m < n ? m : n;
    double R11 = 0.0;
    *r11 = 0.0;
    for (int k = 0; k < steps; ++k) {
        int p = k;
        double best = -1.0;
        for (int c = k; c < n; ++c) {
            double nc = col_norm(A + (size_t)c * lda + k, m - k);
            if (nc > best || (nc == best && perm[c] < perm[p])) {
                best = nc;
                p = c;
            }
        }
        if (p != k) {
            for (int i = 0; i < m; ++i) {
                double t = A[(size_t)k * lda + i];
                A[(size_t)k * lda + i] = A[(size_t)p * lda + i];
                A[(size_t)p * lda + i] = t;
            }
            int t = perm[k];
            perm[k] = perm[p];
            perm[p] = t;
        }
        double *x = A + (size_t)k * lda + k;
        double nx = col_norm(x, m - k);
        if (k == 0) {
            R11 = nx;
            *r11 = nx;
        }
        if (nx == 0.0 || nx < tol * R11) return k;
        double alpha = x[0];
        double beta = alpha >= 0.0 ? -nx : nx;
        double scale = 1.0 / (alpha - beta);
        for (int i = 1; i < m - k; ++i) x[i] *= scale;
        tau[k] = (beta - alpha) / beta;
        x[0] = beta;
        for (int c = k + 1; c < n; ++c) {
            double *a = A + (size_t)c * lda + k;
            double s = a[0];
            for (int i = 1; i < m - k; ++i) s += x[i] * a[i];
            s *= tau[k];
            a[0] -= s;
            for (int i = 1; i < m - k; ++i) a[i] -= s * x[i];
        }
    }
    return steps;
}

/* Q_hat = H_0 H_1 ... H_{r-1} [I_r; 0] (m x r, ld = m): the orthonormal factor
 * of the kept columns, Proposition 3.1. */
void orc_form_q(int m, int r, const double *A, int lda, const double *tau, double *Q) {
    for (int c = 0; c < r; ++c)
        for (int i = 0; i < m; ++i) Q[(size_t)c * m + i] = (i == c) ? 1.0 : 0.0;
    for (int k = r - 1; k >= 0; --k) {
        const double *v = A + (size_t)k * lda + k; /* v[0] = 1 implied */
        for (int c = 0; c < r; ++c) {
            double *q = Q + (size_t)c * m + k;
            double s = q[0];
            for (int i = 1; i < m - k; ++i) s += v[i] * q[i];
            s *= tau[k];
            q[0] -= s;
            for (int i = 1; i < m - k; ++i) q[i] -= s * v[i];
        }
    }
}

/* Solve R z = x in place, R upper triangular r x r (column-major, ldr). */
void orc_trsv_upper(int r, const double *R, int ldr, double *x) {
    for (int i = r - 1; i >= 0; --i) {
        double s = x[i];
        for (int c = i + 1; c < r; ++c) s -= R[(size_t)c * ldr + i] * x[c];
        x[i] = s / R[(size_t)i * ldr + i];
    }
}

/* Solve R^T z = x in place. */
void orc_trsv_upper_t(int r, const double *R, int ldr, double *x) {
    for (int i = 0; i < r; ++i) {
        double s = x[i];
        for (int c = 0; c < i; ++c) s -= R[(size_t)i * ldr + c] * x[c];
        x[i] = s / R[(size_t)i * ldr + i];
    }
}

/* ------------------------------------------------------------------------ */
/* the filtered, right-preconditioned operator and LSQR (Algorithm 2)        */
/* ------------------------------------------------------------------------ */

/* Block system after filtering.  Block j owns rows grow[roff[j] .. roff[j]+m[j])
 * and r[j] kept columns, stored at coff[j] in the compact column vector.
 * Ahat holds M_j[:, kept] (m_j x r_j, ld m_j) at aoff[j]; R holds R_hat_j
 * (r_j x r_j, ld r_j) at Roff[j].
 * mode 0: operator Ahat S^-1 with S^-1 = blockdiag(R_hat_j^-1) (Sec. 3.2);
 * mode 1: operator Ahat (no preconditioner);
 * in both cases Ahat may also be an explicit Q_hat (Proposition 3.1) with mode 1. */
typedef struct {
    int64_t J, N;
    const int64_t *m, *roff, *grow, *coff, *aoff, *Roff;
    const int32_t *r;
    const double *Ahat, *R;
    int32_t mode;
} orc_system;

static int64_t ncols(const orc_system *S) {
    int64_t c = 0;
    for (int64_t j = 0; j < S->J; ++j) c += S->r[j];
    return c;
}

/* out = Op x (out has N entries) */
static void op_apply(const orc_system *S, const double *x, double *out, double *tmp) {
    for (int64_t i = 0; i < S->N; ++i) out[i] = 0.0;
    for (int64_t j = 0; j < S->J; ++j) {
        int rj = S->r[j];
        int64_t mj = S->m[j];
        for (int c = 0; c < rj; ++c) tmp[c] = x[S->coff[j] + c];
        if (S->mode == 0) orc_trsv_upper(rj, S->R + S->Roff[j], rj, tmp);
        const double *A = S->Ahat + S->aoff[j];
        for (int64_t lr = 0; lr < mj; ++lr) {
            double s = 0.0;
            for (int c = 0; c < rj; ++c) s += A[(size_t)c * mj + lr] * tmp[c];
            out[S->grow[S->roff[j] + lr]] += s;
        }
    }
}

/* out = Op^T y (out has sum r_j entries) */
static void op_apply_t(const orc_system *S, const double *y, double *out) {
    for (int64_t j = 0; j < S->J; ++j) {
        int rj = S->r[j];
        int64_t mj = S->m[j];
        const double *A = S->Ahat + S->aoff[j];
        double *o = out + S->coff[j];
        for (int c = 0; c < rj; ++c) {
            double s = 0.0;
            for (int64_t lr = 0; lr < mj; ++lr) s += A[(size_t)c * mj + lr] * y[S->grow[S->roff[j] + lr]];
            o[c] = s;
        }
        if (S->mode == 0) orc_trsv_upper_t(rj, S->R + S->Roff[j], rj, o);
    }
}

void orc_op_apply(const orc_system *S, const double *x, double *out) {
    int64_t maxr = 0;
    for (int64_t j = 0; j < S->J; ++j) if (S->r[j] > maxr) maxr = S->r[j];
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(maxr + 1));
    op_apply(S, x, out, tmp);
    free(tmp);
}

void orc_op_apply_t(const orc_system *S, const double *y, double *out) { op_apply_t(S, y, out); }

static double vnorm(const double *a, int64_t n) { return col_norm(a, n); }

/* LSQR (Paige and Saunders 1982, the bidiagonalisation algorithm with the
 * plane-rotation update of x and w) on min ||Op y - h||.
 * Start: y0 (NULL = zero); the iteration runs on the residual system and adds
 * its result to y0.  Stopping (tests of the 1982 paper, no condition limit):
 *   ||r|| <= btol ||h|| + atol ||Op||_F ||y||       (istop 1)
 *   ||Op^T r|| <= atol ||Op||_F ||r||                (istop 2)
 *   beta_1 = 0 or alpha_1 = 0: y0 is exact          (istop 0)
 *   iteration limit                                  (istop 7)
 * with the norm estimates of the paper: ||r|| = phibar, ||Op^T r|| =
 * phibar alpha |c|, ||Op||_F^2 = sum(alpha_i^2 + beta_{i+1}^2); ||y|| is
 * computed exactly.  stats = {itn, istop, rnorm, arnorm, anorm, ynorm}.
 * rhist (optional, max_iter+1 entries) receives phibar after each iteration. */
int orc_lsqr(const orc_system *S, const double *h, const double *y0, double atol, double btol,
             int max_iter, double *y, double *stats, double *rhist) {
    int64_t N = S->N, n = ncols(S);
    int64_t maxr = 0;
    for (int64_t j = 0; j < S->J; ++j) if (S->r[j] > maxr) maxr = S->r[j];
    double *u = (double *)calloc((size_t)N, sizeof(double));
    double *v = (double *)calloc((size_t)n + 1, sizeof(double));
    double *w = (double *)calloc((size_t)n + 1, sizeof(double));
    double *dx = (double *)calloc((size_t)n + 1, sizeof(double));
    double *t = (double *)calloc((size_t)n + 1, sizeof(double));
    double *tmp = (double *)calloc((size_t)maxr + 1, sizeof(double));
    double *Au = (double *)calloc((size_t)N, sizeof(double));

    if (y0) {
        op_apply(S, y0, Au, tmp);
        for (int64_t i = 0; i < N; ++i) u[i] = h[i] - Au[i];
    } else {
        for (int64_t i = 0; i < N; ++i) u[i] = h[i];
    }
    double bnorm = vnorm(h, N);
    double beta = vnorm(u, N);
    if (beta > 0.0) for (int64_t i = 0; i < N; ++i) u[i] /= beta;
    op_apply_t(S, u, v);
    double alpha = vnorm(v, n);
    if (alpha > 0.0) for (int64_t i = 0; i < n; ++i) v[i] /= alpha;
    for (int64_t i = 0; i < n; ++i) w[i] = v[i];
    double phibar = beta, rhobar = alpha, anorm2 = 0.0;
    double rnorm = beta, arnorm = alpha * beta, anorm = 0.0, ynorm = 0.0;
    int itn = 0, istop = 0;
    if (rhist) rhist[0] = beta;
    if (beta == 0.0 || alpha == 0.0) {
        istop = 0;
    } else {
        istop = 7;
        while (itn < max_iter) {
            ++itn;
            /* bidiagonalisation: beta u = Op v - alpha u ; alpha v = Op^T u - beta v */
            op_apply(S, v, Au, tmp);
            for (int64_t i = 0; i < N; ++i) u[i] = Au[i] - alpha * u[i];
            double beta_n = vnorm(u, N);
            if (beta_n > 0.0) for (int64_t i = 0; i < N; ++i) u[i] /= beta_n;
            anorm2 += alpha * alpha + beta_n * beta_n;
            op_apply_t(S, u, t);
            for (int64_t i = 0; i < n; ++i) v[i] = t[i] - beta_n * v[i];
            double alpha_n = vnorm(v, n);
            if (alpha_n > 0.0) for (int64_t i = 0; i < n; ++i) v[i] /= alpha_n;
            /* plane rotation eliminating beta_{i+1} */
            double rho = sqrt(rhobar * rhobar + beta_n * beta_n);
            double c = rhobar / rho, s = beta_n / rho;
            double theta = s * alpha_n;
            rhobar = -c * alpha_n;
            double phi = c * phibar;
            phibar = s * phibar;
            /* update of the iterate and of the search direction */
            for (int64_t i = 0; i < n; ++i) {
                dx[i] += (phi / rho) * w[i];
                w[i] = v[i] - (theta / rho) * w[i];
            }
            alpha = alpha_n;
            beta = beta_n;
            rnorm = phibar;
            arnorm = phibar * alpha_n * fabs(c);
            anorm = sqrt(anorm2);
            double yn2 = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                double yi = dx[i] + (y0 ? y0[i] : 0.0);
                yn2 += yi * yi;
            }
            ynorm = sqrt(yn2);
            if (rhist) rhist[itn] = phibar;
            if (rnorm <= btol * bnorm + atol * anorm * ynorm) { istop = 1; break; }
            if (arnorm <= atol * anorm * rnorm) { istop = 2; break; }
        }
    }
    for (int64_t i = 0; i < n; ++i) y[i] = dx[i] + (y0 ? y0[i] : 0.0);
    if (stats) {
        stats[0] = itn; stats[1] = istop; stats[2] = rnorm; stats[3] = arnorm;
        stats[4] = anorm; stats[5] = ynorm;
    }
    free(u); free(v); free(w); free(dx); free(t); free(tmp); free(Au);
    return istop;
}

/* Coefficients of Algorithm 2's output: a_j[perm_j[c]] = (R_hat_j^-1 y_j)[c]
 * for kept c < r_j, 0 at dropped columns.  perm holds J*K entries. */
void orc_coefficients(int64_t J, int K, const int32_t *r, const int32_t *perm, const int64_t *coff,
                      const int64_t *Roff, const double *R, const double *y, double *a) {
    double *t = (double *)malloc(sizeof(double) * (size_t)(K + 1));
    for (int64_t j = 0; j < J; ++j) {
        for (int k = 0; k < K; ++k) a[j * K + k] = 0.0;
        for (int c = 0; c < r[j]; ++c) t[c] = y[coff[j] + c];
        orc_trsv_upper(r[j], R + Roff[j], r[j], t);
        for (int c = 0; c < r[j]; ++c) a[j * K + perm[j * K + c]] = t[c];
    }
    free(t);
}

/* ------------------------------------------------------------------------ */
/* evaluation (Eq. (1)) and errors (Sec. 4.2)                                */
/* ------------------------------------------------------------------------ */

/* u_hat(x) = g(x) sum_j w_j(x) sum_k a_jk phi_jk(x) at npts points X
 * (npts x dim), g the hard-constraint factor (1 without one).  The
 * normalising sum W(x) = sum_l hat_w_l(x) is the same for every j at a point,
 * so it is formed once per point (same terms, same order as in orc_window)
 * and w_j = hat_w_j / W. */
void orc_eval(const orc_problem *P, const double *params, const double *a, int64_t npts,
              const double *X, double *u) {
    int64_t J = orc_num_subdomains(P);
    const int64_t np = orc_params_per_subdomain(P);
    const int nl = n_last(P);
    for (int64_t p = 0; p < npts; ++p) {
        double x[3] = {0, 0, 0};
        for (int i = 0; i < P->dim; ++i) x[i] = X[p * P->dim + i];
        double W = 0.0;
        for (int64_t l = 0; l < J; ++l) {
            double dw[3], d2w[3];
            W += orc_window_hat(P, l, x, dw, d2w);
        }
        double s = 0.0;
        for (int64_t j = 0; j < J; ++j) {
            double dw[3], d2w[3];
            double h = orc_window_hat(P, j, x, dw, d2w);
            if (h == 0.0 || W == 0.0) continue;
            double w = h / W;
            double mu[3], sig[3];
            orc_subdomain(P, j, mu, sig);
            double z[ORC_MAXH], dz[3][ORC_MAXH], d2z[3][ORC_MAXH];
            int nin = last_hidden(P, params + j * np, mu, sig, x, z, dz, d2z);
            double sj = 0.0;
            for (int k = 0; k < P->K; ++k) {
                double phi, dphi[3], d2phi[3];
                feature_from(P, params + j * np + (int64_t)k * (nl + 1), nin, z, dz, d2z, &phi, dphi, d2phi);
                sj += a[j * P->K + k] * phi;
            }
            s += w * sj;
        }
        double gd[3], gd2[3];
        u[p] = hard_factor(P, x, gd, gd2) * s;
    }
}

void orc_exact_many(const orc_problem *P, int64_t npts, const double *X, double *u) {
    for (int64_t p = 0; p < npts; ++p) {
        double x[3] = {0, 0, 0};
        for (int i = 0; i < P->dim; ++i) x[i] = X[p * P->dim + i];
        u[p] = orc_exact(P, x);
    }
}

/* ------------------------------------------------------------------------ */
/* feature values (for the local fit of a predicted solution)               */
/* ------------------------------------------------------------------------ */

/* Phi[p, k] = phi_jk(X_p) for the K features of subdomain j (no window), at
 * npts points X (npts x dim); Phi column-major with ld = npts. */
void orc_feature_values(const orc_problem *P, const double *params, int64_t j, int64_t npts, const double *X,
                        double *Phi) {
    double mu[3], sig[3];
    orc_subdomain(P, j, mu, sig);
    const int64_t np = orc_params_per_subdomain(P);
    const int nl = n_last(P);
    for (int64_t p = 0; p < npts; ++p) {
        double x[3] = {0, 0, 0};
        for (int i = 0; i < P->dim; ++i) x[i] = X[p * P->dim + i];
        double z[ORC_MAXH], dz[3][ORC_MAXH], d2z[3][ORC_MAXH];
        int nin = last_hidden(P, params + j * np, mu, sig, x, z, dz, d2z);
        for (int k = 0; k < P->K; ++k) {
            double phi, dphi[3], d2phi[3];
            feature_from(P, params + j * np + (int64_t)k * (nl + 1), nin, z, dz, d2z, &phi, dphi, d2phi);
            Phi[(size_t)k * npts + p] = phi;
        }
    }
}
