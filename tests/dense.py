"""Dense reference matrices for tiny problems, built from the definitions
(test helper; used only to pin the oracle)."""
import math

import numpy as np


def rays_by_definition(g):
    """Source and direction of every ray from the stated fan convention."""
    dg = g.dgamma if g.dgamma > 0 else 2 * math.asin(g.n * g.pixel_mm / math.sqrt(2) / g.dso_mm) / g.n_bins
    out = []
    for v in range(g.n_views):
        b = g.beta0 + g.arc * v / g.n_views
        for j in range(g.n_bins):
            gm = (j - (g.n_bins - 1) / 2) * dg
            out.append(((g.dso_mm * math.cos(b), g.dso_mm * math.sin(b)),
                        (math.cos(b + math.pi + gm), math.sin(b + math.pi + gm))))
    return out


def chord(S, u, xa, xb, ya, yb):
    """Length of the line S + t u inside the rectangle [xa,xb] x [ya,yb]."""
    lo, hi = -math.inf, math.inf
    for s, d, a, b in ((S[0], u[0], xa, xb), (S[1], u[1], ya, yb)):
        if d == 0.0:
            if not (a <= s < b):
                return 0.0
            continue
        t1, t2 = (a - s) / d, (b - s) / d
        lo, hi = max(lo, min(t1, t2)), min(hi, max(t1, t2))
    return max(0.0, hi - lo)


def dense_A(g):
    """System matrix (V*nb, n*n) by clipping every ray against every pixel."""
    n, px = g.n, g.pixel_mm
    x0 = -n * px / 2
    rays = rays_by_definition(g)
    A = np.zeros((len(rays), n * n))
    for r, (S, u) in enumerate(rays):
        for iy in range(n):
            for ix in range(n):
                A[r, iy * n + ix] = chord(S, u, x0 + ix * px, x0 + (ix + 1) * px,
                                          x0 + iy * px, x0 + (iy + 1) * px)
    return A


def ramlak(k):
    """Band-limited ramp tap in bin units (its frequency response |w|/2pi is
    checked separately)."""
    if k == 0:
        return 0.25
    return 0.0 if k % 2 == 0 else -1.0 / (math.pi * math.pi * k * k)


def dense_C(g):
    """Filtration as a block-diagonal matrix: c0 * Toeplitz(h) per view."""
    nb = g.n_bins
    j = np.arange(nb)
    T = np.vectorize(ramlak)(j[:, None] - j[None, :])
    if not g.filter:
        T = np.eye(nb)
    else:
        T = T * math.pi / (g.n_views * g.pixel_mm ** 2)
    return np.kron(np.eye(g.n_views), T)


def dense_W(n):
    """The 9 n^2 x n^2 framelet analysis matrix from the 1-D taps, periodic."""
    s = math.sqrt(2) / 4
    taps = [(0.25, 0.5, 0.25), (s, 0.0, -s), (-0.25, 0.5, -0.25)]
    W = np.zeros((9 * n * n, n * n))
    for a in range(3):
        for b in range(3):
            band = 3 * a + b
            for y in range(n):
                for x in range(n):
                    r = band * n * n + y * n + x
                    for p in (-1, 0, 1):
                        for q in (-1, 0, 1):
                            W[r, ((y + p) % n) * n + (x + q) % n] += taps[a][p + 1] * taps[b][q + 1]
    return W
