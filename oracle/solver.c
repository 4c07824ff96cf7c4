/*
 * Oracle (test infrastructure only): the AIR split-Bregman solve.
 *
 * Objective (Eq. 1 with P = C^{1/2}, Eq. 3, and R = tensor framelet):
 *     min_X  1/2 ||P (A X - Y)||^2 + lambda ||W X||_1.
 * Split Bregman (the paper's ref. [24]) introduces d = W X and alternates
 *   (1) the L2 step, which the paper says is solved like Eq. (5):
 *         (A'^T A + mu I) X = A'^T Y + mu W^T (d - b),   A'^T = A^T C,
 *       using W^T W = I; solved here by n_cg conjugate-gradient steps
 *       warm-started from the current X;
 *   (2) d = S_{lambda/mu}(W X + b) on the high-pass bands, b <- b + W X - d.
 * The 1/2 on the data term and the mu/2 on the split penalty make the
 * threshold lambda/mu and the L2 step exactly the system above.
 * X^0 = 0, b^0 = 0, g^0 = W^T(d^0 - b^0) = 0; fixed n_outer and n_cg, no
 * tolerance stop, no positivity constraint.
 */
#include "orc.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static double dot(const double *a, const double *b, size_t n)
{
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* out = (A^T C A + mu I) x */
static void apply_M(const orc_geom *g, const double *x, double mu, double *out, double *sino)
{
    const size_t np = (size_t)g->n * g->n;
    orc_project(g, x, sino);
    orc_filtered_backproject(g, sino, out);
    for (size_t i = 0; i < np; ++i) out[i] += mu * x[i];
}

/* Conjugate gradients (Hestenes-Stiefel) on the SPD system M X = rhs.
 * Stops early, leaving X as it is, when rho = r.r is 0 or p.Mp <= 0. */
void orc_cg(const orc_geom *g, const double *rhs, double mu, int n_cg, double *X)
{
    const size_t np = (size_t)g->n * g->n;
    double *r = (double *)malloc(sizeof(double) * np);
    double *p = (double *)malloc(sizeof(double) * np);
    double *q = (double *)malloc(sizeof(double) * np);
    double *sino = (double *)malloc(sizeof(double) * (size_t)g->n_views * g->n_bins);

    apply_M(g, X, mu, q, sino);
    for (size_t i = 0; i < np; ++i) r[i] = rhs[i] - q[i];
    memcpy(p, r, sizeof(double) * np);
    double rho = dot(r, r, np);

    for (int it = 0; it < n_cg; ++it) {
        if (rho == 0.0) break;
        apply_M(g, p, mu, q, sino);
        double pq = dot(p, q, np);
        if (!(pq > 0.0)) break;
        double alpha = rho / pq;
        for (size_t i = 0; i < np; ++i) {
            X[i] += alpha * p[i];
            r[i] -= alpha * q[i];
        }
        double rho_new = dot(r, r, np);
        double beta = rho_new / rho;
        for (size_t i = 0; i < np; ++i) p[i] = r[i] + beta * p[i];
        rho = rho_new;
    }
    free(r);
    free(p);
    free(q);
    free(sino);
}

void orc_solve(const orc_geom *g, const double *Y, double lambda, double mu,
               int n_outer, int n_cg, double *X, double *resid)
{
    const int n = g->n;
    const size_t np = (size_t)n * n;
    double *rhs0 = (double *)malloc(sizeof(double) * np);
    double *rhs = (double *)malloc(sizeof(double) * np);
    double *gg = (double *)calloc(np, sizeof(double));
    double *b = (double *)calloc(9 * np, sizeof(double));

    orc_filtered_backproject(g, Y, rhs0);          /* A'^T Y, once */
    for (size_t i = 0; i < np; ++i) X[i] = 0.0;

    for (int k = 0; k < n_outer; ++k) {
        for (size_t i = 0; i < np; ++i) rhs[i] = rhs0[i] + mu * gg[i];
        orc_cg(g, rhs, mu, n_cg, X);
        double r = orc_shrink(n, X, b, gg, lambda / mu);
        if (resid) resid[k] = r;
    }
    free(rhs0);
    free(rhs);
    free(gg);
    free(b);
}
