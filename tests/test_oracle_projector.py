"""Pins of the oracle's geometry, X-ray transform A and transpose A^T.

Everything here is checked against something other than the oracle itself:
slab-clipped chord lengths computed by hand (the definition of a line/box
intersection, a different algorithm from Siddon's merged crossings), a dense
8x8 system matrix built pixel by pixel, the Kak-Slaney closed form of an
ellipse's line integral, and convergence to the analytic phantom.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1310_1434_gb300 import inputs

from dense import chord, dense_A, rays_by_definition


def geom(n, px, V, nb, **kw):
    return oracle.Geometry(n=n, pixel_mm=px, n_views=V, n_bins=nb, **kw)


def test_ray_geometry_matches_definition():
    g = geom(64, 1.3, 7, 33, beta0=0.3, arc=math.pi)
    for k, (S, u) in enumerate(rays_by_definition(g)):
        s, d = oracle.ray(g, k // g.n_bins, k % g.n_bins)
        assert np.allclose(s, S, rtol=0, atol=1e-12) and np.allclose(d, u, rtol=0, atol=1e-15)


def test_auto_fan_covers_circumscribed_circle():
    # the outermost ray edges are tangent to the circle of radius n*dx/sqrt2
    g = geom(512, 0.8, 4, 738)
    dg = oracle.dgamma(g)
    half_fan = dg * g.n_bins / 2
    assert math.isclose(g.dso_mm * math.sin(half_fan), 512 * 0.8 / math.sqrt(2), rel_tol=1e-14)


@pytest.mark.parametrize("n,px,V,nb", [(16, 1.0, 12, 31), (37, 0.7, 9, 40), (64, 1.6, 20, 90)])
def test_all_ones_image_gives_box_chords(n, px, V, nb):
    g = geom(n, px, V, nb)
    Y = oracle.project(g, np.ones((n, n)))
    h = n * px / 2
    exp = np.array([chord(S, u, -h, h, -h, h) for S, u in rays_by_definition(g)]).reshape(V, nb)
    scale = 2 * h * math.sqrt(2)
    assert np.max(np.abs(Y - exp)) <= 1e-10 * scale
    assert (exp > 0).mean() > 0.5  # the fan really does hit the image


def test_rectangle_chords():
    n, px = 40, 1.0
    g = geom(n, px, 15, 64, beta0=0.1)
    X = np.zeros((n, n))
    ix0, ix1, iy0, iy1 = 5, 23, 11, 17        # pixels [ix0,ix1) x [iy0,iy1)
    X[iy0:iy1, ix0:ix1] = 1.0
    Y = oracle.project(g, X)
    x0 = -n * px / 2
    exp = np.array([chord(S, u, x0 + ix0 * px, x0 + ix1 * px, x0 + iy0 * px, x0 + iy1 * px)
                    for S, u in rays_by_definition(g)]).reshape(Y.shape)
    assert np.max(np.abs(Y - exp)) <= 1e-10 * 30
    assert (exp > 0).sum() > 100


G8 = dict(n=8, px=1.25, V=12, nb=16)


def test_dense_8x8_matrix_columns():
    g = geom(G8["n"], G8["px"], G8["V"], G8["nb"])
    A = dense_A(g)
    for i in range(64):
        e = np.zeros(64)
        e[i] = 1.0
        col = oracle.project(g, e.reshape(8, 8)).ravel()
        # FP64 crossing parameters are ~850 mm from the source: a few ulp of that
        assert np.max(np.abs(col - A[:, i])) <= 1e-12
    assert np.count_nonzero(A) > 300


def test_dense_8x8_transpose_rows():
    g = geom(G8["n"], G8["px"], G8["V"], G8["nb"])
    A = dense_A(g)
    for r in range(0, A.shape[0], 7):
        e = np.zeros(A.shape[0])
        e[r] = 1.0
        row = oracle.backproject(g, e.reshape(g.n_views, g.n_bins)).ravel()
        assert np.max(np.abs(row - A[r])) <= 1e-12


@pytest.mark.parametrize("n,px,V,nb,arc", [(32, 1.0, 30, 48, 2 * math.pi), (50, 0.9, 17, 75, 2 * math.pi),
                                           (64, 1.0, 16, 96, math.pi)])
def test_adjoint_identity(n, px, V, nb, arc):
    g = geom(n, px, V, nb, arc=arc)
    rng = np.random.Generator(np.random.PCG64(3))
    x = rng.standard_normal((n, n))
    y = rng.standard_normal((V, nb))
    lhs = float(np.sum(oracle.project(g, x) * y))
    rhs = float(np.sum(x * oracle.backproject(g, y)))
    scale = float(np.sum(np.abs(oracle.project(g, np.abs(x)) * np.abs(y))))
    assert abs(lhs - rhs) <= 1e-12 * scale


def test_fan_orientation():
    # view 0: source on +x, a ray with gamma > 0 heads toward -y; view V/4:
    # source on +y, gamma > 0 heads toward +x.
    n = 32
    g = geom(n, 1.0, 4, 33)
    low = np.zeros((n, n))
    low[2:10, 12:20] = 1.0                  # rows iy 2..9 are at y < 0
    Y = oracle.project(g, low)
    c = (g.n_bins - 1) // 2
    assert Y[0, c + 1:].sum() > 0 and Y[0, :c].sum() == 0
    right = np.zeros((n, n))
    right[12:20, 22:30] = 1.0               # columns ix 22..29 are at x > 0
    Y = oracle.project(g, right)
    assert Y[1, c + 1:].sum() > 0 and Y[1, :c].sum() == 0


def kak_slaney(S, u, e):
    """Line integral of a uniform ellipse via the support-function closed form:
    2 rho a b sqrt(a^2 cos^2 + b^2 sin^2 - s^2) / (a^2 cos^2 + b^2 sin^2), with
    the line written as {x : x.nhat = s} relative to the ellipse centre and the
    angle measured from the ellipse's a-axis."""
    nx, ny = -u[1], u[0]
    th = math.atan2(ny, nx) - e.phi
    s = (S[0] - e.cx) * nx + (S[1] - e.cy) * ny
    a2 = (e.a * math.cos(th)) ** 2 + (e.b * math.sin(th)) ** 2
    if s * s >= a2:
        return 0.0
    return 2 * e.rho * e.a * e.b * math.sqrt(a2 - s * s) / a2


def test_ellipse_generator_matches_closed_form():
    w = inputs.AIR128
    g = inputs.Geometry(64, 2.0, 24, 96)
    ell = inputs.random_phantom(g, 11, 6, 3)
    p = inputs.ellipse_line_integrals(g, ell)
    S, U = inputs.ray_lines(g)
    worst = 0.0
    for v in range(g.n_views):
        for j in range(g.n_bins):
            ref = sum(kak_slaney(S[v, 0], U[v, j], e) for e in ell)
            worst = max(worst, abs(p[v, j] - ref) / max(abs(ref), 1e-3))
    assert worst <= 1e-10
    assert w.geom.n == 128


def test_generator_rays_equal_oracle_rays():
    g = inputs.Geometry(48, 1.1, 10, 70, beta0=0.2)
    S, U = inputs.ray_lines(g)
    og = oracle.Geometry(**{k: getattr(g, k) for k in oracle.Geometry.__dataclass_fields__})
    for v in range(g.n_views):
        for j in range(0, g.n_bins, 9):
            s, u = oracle.ray(og, v, j)
            assert np.allclose(s, S[v, 0], atol=1e-12) and np.allclose(u, U[v, j], atol=1e-14)


def test_siddon_converges_to_analytic_phantom():
    # Same rays, finer and finer pixels over the same field of view: A applied
    # to the rasterised phantom tends to the exact line integrals.
    fov = 128.0
    errs = []
    for n in (32, 64, 128):
        gi = inputs.Geometry(n, fov / n, 18, 64, dgamma=0.0012)
        ell = [inputs.Ellipse(10.0, -6.0, 35.0, 20.0, 0.4, 0.02),
               inputs.Ellipse(-20.0, 15.0, 12.0, 12.0, 0.0, 0.01)]
        exact = inputs.ellipse_line_integrals(gi, ell)
        X = inputs.rasterize(gi, ell, ss=8)
        og = oracle.Geometry(**{k: getattr(gi, k) for k in oracle.Geometry.__dataclass_fields__})
        errs.append(np.linalg.norm(oracle.project(og, X) - exact) / np.linalg.norm(exact))
    assert errs[0] < 0.05
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 0.45 * errs[0]
