/*
 * mlp_oracle.c -- plain FP64 loops for the warm-start network: forward pass,
 * mean-squared-error loss, its gradient by backpropagation, and one Adam step.
 *
 * TEST INFRASTRUCTURE ONLY, like rfm_oracle.c: the CUDA library is checked
 * against these functions and never calls them.
 *
 * The paper has no network of its own here; the definitions are the textbook
 * ones, written out sample by sample with no batching into matrix products:
 *   - fully connected network with widths w[0..L]: layer l (1..L) forms
 *     z_l = W_l h_{l-1} + b_l from h_0 = x, then h_l = tanh(z_l) for l < L and
 *     h_L = z_L (linear output);
 *   - loss over a batch of B samples: (1/B) sum_i (h_L(x_i) - t_i)^2;
 *   - gradient by the chain rule (backpropagation): the output error is
 *     e_L = 2 (h_L - t) / B, dW_l = sum_i e_l h_{l-1}^T, db_l = sum_i e_l, and
 *     e_{l-1} = (W_l^T e_l) * (1 - h_{l-1}^2);
 *   - Adam (Kingma and Ba 2015, Algorithm 1): first and second moment
 *     estimates with bias correction.
 * Parameters are packed layer by layer: W_l row-major (w[l] rows of w[l-1]),
 * then b_l.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int64_t orc_mlp_nparams(int L, const int *w) {
    int64_t n = 0;
    for (int l = 1; l <= L; ++l) n += (int64_t)w[l] * w[l - 1] + w[l];
    return n;
}

static int max_width(int L, const int *w) {
    int m = 0;
    for (int l = 0; l <= L; ++l)
        if (w[l] > m) m = w[l];
    return m;
}

/* activations of one sample: h[l] for l = 0..L, each of width w[l] */
static void forward_one(int L, const int *w, const double *theta, const double *x, double **h) {
    for (int i = 0; i < w[0]; ++i) h[0][i] = x[i];
    const double *p = theta;
    for (int l = 1; l <= L; ++l) {
        const int no = w[l], ni = w[l - 1];
        const double *W = p, *b = p + (int64_t)no * ni;
        for (int o = 0; o < no; ++o) {
            double z = b[o];
            for (int i = 0; i < ni; ++i) z += W[(int64_t)o * ni + i] * h[l - 1][i];
            h[l][o] = l < L ? tanh(z) : z;
        }
        p += (int64_t)no * ni + no;
    }
}

static double **alloc_acts(int L, const int *w) {
    double **h = (double **)malloc(sizeof(double *) * (L + 1));
    for (int l = 0; l <= L; ++l) h[l] = (double *)calloc((size_t)w[l], sizeof(double));
    return h;
}

static void free_acts(int L, double **h) {
    for (int l = 0; l <= L; ++l) free(h[l]);
    free(h);
}

/* Y[i] = network output for sample i (X row-major B x w[0]); w[L] must be 1 */
void orc_mlp_forward(int L, const int *w, const double *theta, int64_t B, const double *X, double *Y) {
    double **h = alloc_acts(L, w);
    for (int64_t s = 0; s < B; ++s) {
        forward_one(L, w, theta, X + s * w[0], h);
        Y[s] = h[L][0];
    }
    free_acts(L, h);
}

/* Loss of the batch and its gradient with respect to every parameter
 * (grad has orc_mlp_nparams entries, overwritten). */
double orc_mlp_grad(int L, const int *w, const double *theta, int64_t B, const double *X, const double *T,
                    double *grad) {
    const int64_t np = orc_mlp_nparams(L, w);
    memset(grad, 0, sizeof(double) * (size_t)np);
    double **h = alloc_acts(L, w);
    const int mw = max_width(L, w);
    double *e = (double *)calloc((size_t)mw, sizeof(double));
    double *en = (double *)calloc((size_t)mw, sizeof(double));
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (L + 1));
    off[1] = 0;
    for (int l = 2; l <= L; ++l) off[l] = off[l - 1] + (int64_t)w[l - 1] * w[l - 2] + w[l - 1];
    double loss = 0.0;
    for (int64_t s = 0; s < B; ++s) {
        forward_one(L, w, theta, X + s * w[0], h);
        const double d = h[L][0] - T[s];
        loss += d * d;
        e[0] = 2.0 * d / (double)B;
        for (int l = L; l >= 1; --l) {
            const int no = w[l], ni = w[l - 1];
            const double *W = theta + off[l];
            double *gW = grad + off[l], *gb = grad + off[l] + (int64_t)no * ni;
            for (int o = 0; o < no; ++o) {
                for (int i = 0; i < ni; ++i) gW[(int64_t)o * ni + i] += e[o] * h[l - 1][i];
                gb[o] += e[o];
            }
            if (l > 1) {
                for (int i = 0; i < ni; ++i) {
                    double t = 0.0;
                    for (int o = 0; o < no; ++o) t += W[(int64_t)o * ni + i] * e[o];
                    en[i] = t * (1.0 - h[l - 1][i] * h[l - 1][i]);
                }
                for (int i = 0; i < ni; ++i) e[i] = en[i];
            }
        }
    }
    free(off);
    free(en);
    free(e);
    free_acts(L, h);
    return loss / (double)B;
}

/* One Adam step at step number t >= 1 (moments m, v updated in place). */
void orc_adam_step(int64_t n, double *theta, double *m, double *v, const double *g, int t, double lr, double b1,
                   double b2, double eps) {
    const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        const double mh = m[i] / c1, vh = v[i] / c2;
        theta[i] -= lr * mh / (sqrt(vh) + eps);
    }
}
