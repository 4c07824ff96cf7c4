/*
 * Oracle (test infrastructure only): the tensor-framelet regulariser
 * R(X) = ||W X||_1 of Eq. (1) and the soft-shrink / Bregman update of the
 * split Bregman loop (Methods section; the paper's refs. [13,15,24]).
 *
 * The paper names the tensor framelet but not its filters; the reading used
 * here is the undecimated one-level piecewise-linear B-spline framelet, whose
 * one-dimensional filters (taps at offsets -1, 0, +1) are
 *     h0 = [1, 2, 1]/4,   h1 = (sqrt 2 / 4)[1, 0, -1],   h2 = [-1, 2, -1]/4,
 * and whose nine 2-D bands are the tensor products h_a (along y) x h_b
 * (along x), band index 3a + b, with periodic boundaries:
 *     (W_ab X)[y][x] = sum_{p,q} h_a[p] h_b[q] X[(y+p) mod n][(x+q) mod n].
 * |H0|^2 + |H1|^2 + |H2|^2 = 1 on the unit circle, so W^T W = I exactly.
 */
#include "orc.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* tap of 1-D filter a at offset p in {-1, 0, 1} */
static double tap(int a, int p)
{
    static const double h0[3] = {0.25, 0.5, 0.25};
    static const double h2[3] = {-0.25, 0.5, -0.25};
    if (a == 0) return h0[p + 1];
    if (a == 2) return h2[p + 1];
    double s = sqrt(2.0) / 4.0;
    return p == -1 ? s : (p == 1 ? -s : 0.0);
}

static int wrap(int i, int n) { return ((i % n) + n) % n; }

void orc_framelet(int n, const double *X, double *coef)
{
    const size_t np = (size_t)n * n;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double *c = coef + (size_t)(3 * a + b) * np;
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x) {
                    double acc = 0.0;
                    for (int p = -1; p <= 1; ++p)
                        for (int q = -1; q <= 1; ++q)
                            acc += tap(a, p) * tap(b, q) * X[wrap(y + p, n) * n + wrap(x + q, n)];
                    c[(size_t)y * n + x] = acc;
                }
        }
}

/* W^T: the adjoint of the correlation above is the convolution
 * X[y][x] = sum_band sum_{p,q} h_a[p] h_b[q] c_band[(y-p) mod n][(x-q) mod n]. */
void orc_framelet_adjoint(int n, const double *coef, double *X)
{
    const size_t np = (size_t)n * n;
    for (size_t i = 0; i < np; ++i) X[i] = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const double *c = coef + (size_t)(3 * a + b) * np;
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x) {
                    double acc = 0.0;
                    for (int p = -1; p <= 1; ++p)
                        for (int q = -1; q <= 1; ++q)
                            acc += tap(a, p) * tap(b, q) * c[wrap(y - p, n) * n + wrap(x - q, n)];
                    X[(size_t)y * n + x] += acc;
                }
        }
}

/* soft threshold S_tau(t) = sign(t) max(|t| - tau, 0), with sign(0) = 0 */
double orc_soft(double t, double tau)
{
    double m = fabs(t) - tau;
    if (m <= 0.0) return 0.0;
    return t > 0.0 ? m : -m;
}

/* One d/b update of split Bregman (Goldstein & Osher, the paper's ref. [24]):
 *   t = W X + b,  d = S_tau(t) (band 0, the low-pass band, is not shrunk),
 *   b <- t - d  (= b + W X - d),  g = W^T (d - b_new).
 * Returns ||W X - d||_2. */
double orc_shrink(int n, const double *X, double *b, double *g, double tau)
{
    const size_t np = (size_t)n * n, nc = 9 * np;
    double *t = (double *)malloc(sizeof(double) * nc);
    double *e = (double *)malloc(sizeof(double) * nc);
    orc_framelet(n, X, t);
    double r2 = 0.0;
    for (size_t i = 0; i < nc; ++i) {
        double wx = t[i];
        double ti = wx + b[i];
        double d = i < np ? ti : orc_soft(ti, tau);
        b[i] = ti - d;
        e[i] = d - b[i];
        r2 += (wx - d) * (wx - d);
    }
    orc_framelet_adjoint(n, e, g);
    free(t);
    free(e);
    return sqrt(r2);
}
