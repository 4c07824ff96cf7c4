/*
 * Oracle (test infrastructure only): the AR filtration C of Eq. (2) and the
 * filtered adjoint A'^T = A^T C of Eq. (5).
 *
 * The paper takes FBP as the analytical method A^{-1} = B C and uses only its
 * filtration C, which it notes is diagonal in the Fourier domain (Eq. 2), so
 * that C is symmetric and P = C^{1/2} exists (Eq. 3).  The filter itself is
 * not written out in the paper; the reading used here is the band-limited
 * Ram-Lak ramp in detector-bin units,
 *     h[0] = 1/4,   h[k] = -1/(pi^2 k^2) for odd k,   h[k] = 0 for even k != 0,
 * applied along the bins of each view as a LINEAR (zero-padded) convolution,
 * scaled by c0 = pi / (n_views * dx^2) so that A^T C A is close to the
 * identity on the image (a discrete FBP over a full rotation).  No apodising
 * window and no fan pre-weighting, which would make C non-symmetric.
 *
 * The convolution is computed with a radix-2 FFT of this file's own: each
 * view is zero-padded to L = 2^ceil(log2(2 n_b - 1)) samples, multiplied by
 * the DFT of the spatial kernel h[k], |k| <= n_b - 1, placed circularly, and
 * the first n_b outputs of the inverse transform are kept.  Because L covers
 * the full linear support, this equals the Toeplitz product Z = c0 Y T with
 * T_{jk} = h[j - k] up to rounding.
 */
#include "orc.h"

#include <math.h>
#include <stdlib.h>

double orc_ramp_tap(int k)
{
    if (k == 0) return 0.25;
    if (k % 2 == 0) return 0.0;
    return -1.0 / (M_PI * M_PI * (double)k * (double)k);
}

double orc_ramp_scale(const orc_geom *g)
{
    return M_PI / ((double)g->n_views * g->pixel_mm * g->pixel_mm);
}

/* In-place iterative radix-2 Cooley-Tukey DFT of length L (a power of two);
 * sign = -1 forward, +1 inverse (unnormalised). */
static void fft(double *re, double *im, int L, int sign)
{
    for (int i = 1, j = 0; i < L; ++i) {          /* bit-reversal permutation */
        int bit = L >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    for (int len = 2; len <= L; len <<= 1) {      /* butterflies */
        double ang = sign * 2.0 * M_PI / len;
        for (int i = 0; i < L; i += len)
            for (int k = 0; k < len / 2; ++k) {
                double wr = cos(ang * k), wi = sin(ang * k);
                int a = i + k, b = i + k + len / 2;
                double xr = re[b] * wr - im[b] * wi;
                double xi = re[b] * wi + im[b] * wr;
                re[b] = re[a] - xr; im[b] = im[a] - xi;
                re[a] += xr;        im[a] += xi;
            }
    }
}

void orc_filter(const orc_geom *g, const double *Y, double *Z)
{
    const int V = g->n_views, B = g->n_bins;
    if (!g->filter) {                             /* IR: C = I */
        for (size_t i = 0; i < (size_t)V * B; ++i) Z[i] = Y[i];
        return;
    }
    int L = 1;
    while (L < 2 * B - 1) L <<= 1;
    const double c0 = orc_ramp_scale(g);

    /* DFT of the kernel, placed circularly: h[k] at k, h[-k] at L - k */
    double *hr = (double *)calloc(L, sizeof(double));
    double *hi = (double *)calloc(L, sizeof(double));
    for (int k = 0; k < B; ++k) {
        hr[k] = orc_ramp_tap(k);
        if (k > 0) hr[L - k] = orc_ramp_tap(-k);
    }
    fft(hr, hi, L, -1);

#pragma omp parallel
    {
        double *re = (double *)malloc(sizeof(double) * L);
        double *im = (double *)malloc(sizeof(double) * L);
#pragma omp for
        for (int v = 0; v < V; ++v) {
            for (int k = 0; k < L; ++k) {
                re[k] = k < B ? Y[(size_t)v * B + k] : 0.0;
                im[k] = 0.0;
            }
            fft(re, im, L, -1);
            for (int k = 0; k < L; ++k) {
                double a = re[k] * hr[k] - im[k] * hi[k];
                double b = re[k] * hi[k] + im[k] * hr[k];
                re[k] = a;
                im[k] = b;
            }
            fft(re, im, L, +1);
            for (int j = 0; j < B; ++j) Z[(size_t)v * B + j] = c0 * re[j] / L;
        }
        free(re);
        free(im);
    }
    free(hr);
    free(hi);
}

/* A'^T Y = A^T (C Y): the filtration step followed by the adjoint X-ray
 * transform (Eqs. 5 and 6). */
void orc_filtered_backproject(const orc_geom *g, const double *Y, double *X)
{
    size_t m = (size_t)g->n_views * g->n_bins;
    double *Z = (double *)malloc(sizeof(double) * m);
    orc_filter(g, Y, Z);
    orc_backproject(g, Z, X);
    free(Z);
}
