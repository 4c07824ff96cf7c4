/*
 * Oracle (test infrastructure only): fan-beam geometry, the X-ray transform
 * A by Siddon's method, and its explicit transpose A^T, in double precision.
 *
 * A is the system matrix of Eq. (1): Y_{v,j} = sum_i l_{ij} X_i, where l_{ij}
 * is the length (mm) of the intersection of ray (v,j) with pixel i.  The
 * paper computes A and A^T on the GPU with the algorithms of its ref. [26]
 * (Materials section); here they are written from the definition.
 *
 * Siddon's method: the ray crosses the x-planes x0 + k*dx and the y-planes
 * x0 + k*dx at parameters t; the sorted list of those crossings inside the
 * image box cuts the ray into segments, each inside one pixel.  The pixel of
 * a segment is the one containing its midpoint (pixels are half-open, so a
 * ray running exactly along a grid line is charged to the pixel on its +
 * side), its length is the difference of its two end parameters, and
 * zero-length segments are dropped.
 */
#include "orc.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Bin pitch: given, or the fan that covers the circumscribed circle. */
double orc_dgamma(const orc_geom *g)
{
    if (g->dgamma > 0.0) return g->dgamma;
    double r = g->n * g->pixel_mm / sqrt(2.0);   /* circumscribed radius */
    return 2.0 * asin(r / g->dso_mm) / g->n_bins;
}

/* Source position and unit direction of ray (v, j). */
void orc_ray(const orc_geom *g, int v, int j, double src[2], double dir[2])
{
    double beta  = g->beta0 + g->arc * (double)v / (double)g->n_views;
    double gamma = ((double)j - 0.5 * (g->n_bins - 1)) * orc_dgamma(g);
    double theta = beta + M_PI + gamma;
    src[0] = g->dso_mm * cos(beta);
    src[1] = g->dso_mm * sin(beta);
    dir[0] = cos(theta);
    dir[1] = sin(theta);
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Parameter interval [lo, hi] of the slab [a, b] along one axis for the line
 * s + t*d; returns 0 when the line misses the slab. */
static int slab(double s, double d, double a, double b, double *lo, double *hi)
{
    if (d == 0.0) {
        if (s < a || s >= b) return 0;
        *lo = -INFINITY;
        *hi = INFINITY;
        return 1;
    }
    double ta = (a - s) / d, tb = (b - s) / d;
    *lo = ta < tb ? ta : tb;
    *hi = ta < tb ? tb : ta;
    return 1;
}

int orc_ray_segments(const orc_geom *g, int v, int j, int *pix, double *len, int cap)
{
    const int n = g->n;
    const double dx = g->pixel_mm, x0 = -0.5 * n * dx, x1 = x0 + n * dx;
    double S[2], u[2];
    orc_ray(g, v, j, S, u);

    double lox, hix, loy, hiy;
    if (!slab(S[0], u[0], x0, x1, &lox, &hix)) return 0;
    if (!slab(S[1], u[1], x0, x1, &loy, &hiy)) return 0;
    double tin = lox > loy ? lox : loy;
    double tout = hix < hiy ? hix : hiy;
    if (!(tout > tin)) return 0;

    /* every plane crossing strictly inside (tin, tout), plus both ends */
    double *t = (double *)malloc(sizeof(double) * (2 * (n + 1) + 2));
    int m = 0;
    t[m++] = tin;
    t[m++] = tout;
    for (int k = 0; k <= n; ++k) {
        double p = x0 + k * dx;
        if (u[0] != 0.0) {
            double tk = (p - S[0]) / u[0];
            if (tk > tin && tk < tout) t[m++] = tk;
        }
        if (u[1] != 0.0) {
            double tk = (p - S[1]) / u[1];
            if (tk > tin && tk < tout) t[m++] = tk;
        }
    }
    qsort(t, m, sizeof(double), cmp_double);

    int cnt = 0;
    for (int s = 0; s + 1 < m; ++s) {
        double l = t[s + 1] - t[s];
        if (!(l > 0.0)) continue;
        double tm = 0.5 * (t[s] + t[s + 1]);
        int ix = (int)floor((S[0] + tm * u[0] - x0) / dx);
        int iy = (int)floor((S[1] + tm * u[1] - x0) / dx);
        if (ix < 0 || ix >= n || iy < 0 || iy >= n) continue;
        if (cnt < cap) {
            pix[cnt] = iy * n + ix;
            len[cnt] = l;
        }
        ++cnt;
    }
    free(t);
    return cnt;
}

double orc_project_ray(const orc_geom *g, const double *X, int v, int j)
{
    int cap = 4 * g->n + 8;
    int *pix = (int *)malloc(sizeof(int) * cap);
    double *len = (double *)malloc(sizeof(double) * cap);
    int m = orc_ray_segments(g, v, j, pix, len, cap);
    double acc = 0.0;
    for (int s = 0; s < m && s < cap; ++s) acc += len[s] * X[pix[s]];
    free(pix);
    free(len);
    return acc;
}

/* Y = A X, one ray at a time. */
void orc_project(const orc_geom *g, const double *X, double *Y)
{
    const int V = g->n_views, B = g->n_bins;
#pragma omp parallel for schedule(dynamic, 1)
    for (int v = 0; v < V; ++v)
        for (int j = 0; j < B; ++j)
            Y[(size_t)v * B + j] = orc_project_ray(g, X, v, j);
}

/* X = A^T Y: every ray scatters Y_{v,j} times its segment lengths into the
 * pixels it crosses; the very same segments as orc_project, so this is the
 * transpose of A by construction.  Each thread owns a private image; the
 * images are summed at the end. */
void orc_backproject(const orc_geom *g, const double *Y, double *X)
{
    const int n = g->n, V = g->n_views, B = g->n_bins;
    const size_t np = (size_t)n * n;
    int nt = orc_threads();
    double *priv = (double *)calloc((size_t)nt * np, sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *img = priv + (size_t)tid * np;
        int cap = 4 * n + 8;
        int *pix = (int *)malloc(sizeof(int) * cap);
        double *len = (double *)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 1)
        for (int v = 0; v < V; ++v)
            for (int j = 0; j < B; ++j) {
                double y = Y[(size_t)v * B + j];
                int m = orc_ray_segments(g, v, j, pix, len, cap);
                for (int s = 0; s < m && s < cap; ++s) img[pix[s]] += len[s] * y;
            }
        free(pix);
        free(len);
    }
    for (size_t i = 0; i < np; ++i) {
        double acc = 0.0;
        for (int t = 0; t < nt; ++t) acc += priv[(size_t)t * np + i];
        X[i] = acc;
    }
    free(priv);
}
