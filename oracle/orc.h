/*
 * FP64 CPU oracle for AIR (fused Analytical and Iterative Reconstruction,
 * Yang, Gao, Qi & Gao, arXiv 1310.1434).
 *
 * THIS IS TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or constant with the CUDA library: every
 * quantity below (ray geometry, Siddon lengths, filter taps, framelet taps,
 * solver steps) is computed here from its definition, in double precision,
 * plainly and slowly.
 *
 * Conventions (the paper leaves them open; they are the readings listed in
 * the design notes):
 *   image   X[iy*n + ix], pixel (ix,iy) covers [x0+ix*dx, x0+(ix+1)*dx) x
 *           [x0+iy*dx, x0+(iy+1)*dx), x0 = -n*dx/2, centred on the isocentre
 *   sinogram Y[v*n_bins + j]
 *   view v  : beta_v = beta0 + arc*v/n_views, source S_v = dso*(cos b, sin b)
 *   bin j   : gamma_j = (j - (n_bins-1)/2)*dgamma, ray direction at angle
 *             beta_v + pi + gamma_j (the central ray -S_v/|S_v| turned
 *             counter-clockwise by gamma_j); the ray is the whole line.
 *   dgamma  : 0 selects 2*asin(n*dx/(sqrt(2)*dso))/n_bins, a fan that just
 *             covers the circle circumscribing the image.
 */
#ifndef ORC_H
#define ORC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int    n;          /* image side N */
    double pixel_mm;   /* pixel pitch dx (mm) */
    int    n_views;    /* V */
    int    n_bins;     /* detector bins n_b */
    double dso_mm;     /* source to isocentre */
    double dsd_mm;     /* source to detector (fixes only the physical bin size) */
    double dgamma;     /* bin angular pitch (rad); 0 = automatic */
    double beta0;      /* first view angle (rad) */
    double arc;        /* angular range covered by the views (rad) */
    int    filter;     /* 1: Ram-Lak filtration C (AIR); 0: C = I (IR) */
} orc_geom;

/* ---- geometry (Materials section: fan-beam MVCT geometry) ---- */
double orc_dgamma(const orc_geom *g);
void   orc_ray(const orc_geom *g, int v, int j, double src[2], double dir[2]);

/* ---- X-ray transform A and its explicit transpose (Eq. 1, Eq. 5) ---- */
/* Segments of one ray through the pixel grid (Siddon's method).  Writes at
 * most cap (pixel index, length) pairs and returns how many it found. */
int    orc_ray_segments(const orc_geom *g, int v, int j, int *pix, double *len, int cap);
double orc_project_ray(const orc_geom *g, const double *X, int v, int j);
void   orc_project(const orc_geom *g, const double *X, double *Y);
void   orc_backproject(const orc_geom *g, const double *Y, double *X);

/* ---- filtration C and the filtered adjoint A'^T = A^T C (Eqs. 2-5) ---- */
double orc_ramp_tap(int k);             /* Ram-Lak tap h[k] in bin units */
double orc_ramp_scale(const orc_geom *g);
void   orc_filter(const orc_geom *g, const double *Y, double *Z);
void   orc_filtered_backproject(const orc_geom *g, const double *Y, double *X);

/* ---- tensor framelet W (piecewise-linear, 1 level, periodic) ---- */
void   orc_framelet(int n, const double *X, double *coef);         /* coef[9][n][n] */
void   orc_framelet_adjoint(int n, const double *coef, double *X);
double orc_soft(double t, double tau);
/* Split-Bregman d/b update: t = WX + b; d = soft(t, tau) on bands 1..8,
 * d = t on band 0; b <- t - d; g = W^T (d - b).  Returns ||WX - d||_2. */
double orc_shrink(int n, const double *X, double *b, double *g, double tau);

/* ---- the solver: split Bregman with a CG-solved L2 step ---- */
/* (A^T C A + mu I) X = rhs by n_cg conjugate-gradient steps from X. */
void   orc_cg(const orc_geom *g, const double *rhs, double mu, int n_cg, double *X);
/* Full AIR split-Bregman solve.  X (n*n) is output only (starts from 0).
 * resid (n_outer, may be NULL) receives ||WX - d||_2 after each outer step. */
void   orc_solve(const orc_geom *g, const double *Y, double lambda, double mu,
                 int n_outer, int n_cg, double *X, double *resid);

/* number of OpenMP threads the oracle will use (1 when built without it) */
int    orc_threads(void);

#ifdef __cplusplus
}
#endif
#endif
