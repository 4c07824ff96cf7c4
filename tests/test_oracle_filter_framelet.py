"""Pins of the oracle's filtration C (Eq. 2), the tensor framelet W and the
soft shrink, against closed forms and textbook identities."""
import math

import numpy as np
import pytest

import oracle


def geom(n, px, V, nb, **kw):
    return oracle.Geometry(n=n, pixel_mm=px, n_views=V, n_bins=nb, **kw)


# ------------------------------------------------------------------ filter C

@pytest.mark.parametrize("w", [0.0, 0.3, 1.0, 2.0, 3.0, -1.7])
def test_ramp_taps_have_ramp_frequency_response(w):
    # sum_k h[k] e^{-i w k} = |w| / (2 pi) on [-pi, pi]: the band-limited ramp.
    # A wrong sign, a dropped pi^2 or a tap on even k all break this.
    K = 200001
    k = np.arange(1, K + 1, 2, dtype=np.float64)
    h_odd = np.array([oracle.ramp_tap(int(i)) for i in k[:50]])
    assert np.allclose(h_odd, -1.0 / (math.pi**2 * k[:50] ** 2), rtol=1e-15)
    assert oracle.ramp_tap(0) == 0.25
    assert all(oracle.ramp_tap(e) == 0.0 for e in (2, 4, -6, 100))
    assert all(oracle.ramp_tap(-i) == oracle.ramp_tap(i) for i in (1, 3, 5, 77))
    resp = 0.25 + 2.0 * np.sum(-1.0 / (math.pi**2 * k**2) * np.cos(w * k))
    assert abs(resp - abs(w) / (2 * math.pi)) < 2e-6


def toeplitz(nb):
    j = np.arange(nb)
    return np.vectorize(oracle.ramp_tap)(j[:, None] - j[None, :])


@pytest.mark.parametrize("V,nb", [(5, 192), (3, 738), (4, 17), (2, 1)])
def test_fft_filter_equals_toeplitz_product(V, nb):
    g = geom(64, 0.8, V, nb)
    rng = np.random.Generator(np.random.PCG64(5))
    Y = rng.standard_normal((V, nb))
    T = toeplitz(nb)
    ref = oracle.ramp_scale(g) * Y @ T
    Z = oracle.filter(g, Y)
    assert np.max(np.abs(Z - ref)) <= 1e-12 * np.max(np.abs(ref)) + 1e-300


def test_filter_scale_and_identity_mode():
    g = geom(100, 0.5, 40, 64)
    assert math.isclose(oracle.ramp_scale(g), math.pi / (40 * 0.25), rel_tol=1e-15)
    Y = np.random.Generator(np.random.PCG64(1)).random((40, 64))
    g.filter = 0
    assert np.array_equal(oracle.filter(g, Y), Y)


def test_filter_is_symmetric_positive_definite():
    T = toeplitz(96)
    assert np.array_equal(T, T.T)
    np.linalg.cholesky(T)                       # raises if not positive definite
    g = geom(32, 1.0, 3, 96)
    rng = np.random.Generator(np.random.PCG64(9))
    y, z = rng.standard_normal((3, 96)), rng.standard_normal((3, 96))
    a, b = np.sum(oracle.filter(g, y) * z), np.sum(y * oracle.filter(g, z))
    assert abs(a - b) <= 1e-12 * np.sum(np.abs(y)) * np.sum(np.abs(z))


def test_filtered_adjoint_is_an_approximate_inverse():
    # A'^T A = A^T C A should act like FBP: close to the identity on a smooth
    # object well inside the field of view.  This pins only the scale c0.
    n, px = 96, 1.0
    g = geom(n, px, 360, 160)
    x0 = -n * px / 2
    c = (np.arange(n) + 0.5) * px + x0
    yy, xx = np.meshgrid(c, c, indexing="ij")
    X = np.exp(-(xx**2 + yy**2) / (2 * 14.0**2))
    R = oracle.filtered_backproject(g, oracle.project(g, X))
    inner = xx**2 + yy**2 < 30.0**2
    rel = np.linalg.norm((R - X)[inner]) / np.linalg.norm(X[inner])
    assert rel < 0.05, rel


# ------------------------------------------------------------------ framelet W

def filter_symbol(a, w):
    taps = {0: (0.25, 0.5, 0.25), 1: (math.sqrt(2) / 4, 0.0, -math.sqrt(2) / 4), 2: (-0.25, 0.5, -0.25)}[a]
    return sum(t * np.exp(-1j * w * p) for t, p in zip(taps, (-1, 0, 1)))


def test_framelet_unitary_extension_principle():
    # the 1-D filters the oracle uses (read back from W on a delta) satisfy
    # |H0|^2 + |H1|^2 + |H2|^2 = 1, the tight-frame condition
    n = 9
    d = np.zeros((n, n))
    d[4, 4] = 1.0
    c = oracle.framelet(d)
    for a in range(3):
        # band (a, 0) applied to a delta: (W_a0 d)[y][x] = h_a[4 - y] h_0[4 - x]
        col = c[3 * a + 0][:, 4] / 0.5
        taps = (col[5], col[4], col[3])      # offsets -1, 0, +1
        ref = {0: (0.25, 0.5, 0.25), 1: (math.sqrt(2) / 4, 0.0, -math.sqrt(2) / 4), 2: (-0.25, 0.5, -0.25)}[a]
        assert np.allclose(taps, ref, atol=1e-16)
    w = np.linspace(-math.pi, math.pi, 101)
    tot = sum(np.abs(filter_symbol(a, w)) ** 2 for a in range(3))
    assert np.allclose(tot, 1.0, atol=1e-15)


@pytest.mark.parametrize("n", [4, 7, 16])
def test_framelet_perfect_reconstruction_and_parseval(n):
    X = np.random.Generator(np.random.PCG64(n)).standard_normal((n, n))
    c = oracle.framelet(X)
    assert c.shape == (9, n, n)
    assert np.max(np.abs(oracle.framelet_adjoint(c) - X)) <= 1e-14 * np.max(np.abs(X)) * 10
    assert math.isclose(np.linalg.norm(c), np.linalg.norm(X), rel_tol=1e-14)


def test_framelet_adjoint_is_transpose():
    n = 6
    rng = np.random.Generator(np.random.PCG64(2))
    X, c = rng.standard_normal((n, n)), rng.standard_normal((9, n, n))
    assert abs(np.sum(oracle.framelet(X) * c) - np.sum(X * oracle.framelet_adjoint(c))) < 1e-12


def test_framelet_closed_forms():
    n = 12
    const = np.full((n, n), 3.5)
    c = oracle.framelet(const)
    assert np.allclose(c[0], 3.5, atol=1e-15) and np.allclose(c[1:], 0.0, atol=1e-15)
    # linear ramp in x (slope s): band (0,1) = (sqrt2/4)(X[x-1] - X[x+1]) = -(sqrt2/2) s
    s = 0.7
    ramp = np.tile(s * np.arange(n, dtype=float), (n, 1))
    c = oracle.framelet(ramp)
    assert np.allclose(c[1][:, 1:-1], -math.sqrt(2) / 2 * s, atol=1e-14)
    assert np.allclose(c[2][:, 1:-1], 0.0, atol=1e-14)           # second difference
    assert np.allclose(c[3][:, 1:-1], 0.0, atol=1e-14)           # y-derivative
    # delta: band (1,1) at (y0-1, x0-1) is h1[+1] h1[+1] = 1/8; at (y0-1, x0+1) it is h1[+1] h1[-1]
    d = np.zeros((n, n))
    d[5, 6] = 1.0
    c = oracle.framelet(d)
    assert math.isclose(c[4][4, 5], 0.125, rel_tol=1e-15)
    assert math.isclose(c[4][4, 7], -0.125, rel_tol=1e-15)
    assert math.isclose(c[8][6, 6], -0.125, rel_tol=1e-15)       # h2[-1] h2[0]


# ------------------------------------------------------------------ shrink

def test_soft_threshold_hand_values():
    assert oracle.soft(0.0, 0.1) == 0.0
    assert oracle.soft(0.05, 0.1) == 0.0 and oracle.soft(-0.05, 0.1) == 0.0
    assert oracle.soft(0.1, 0.1) == 0.0 and oracle.soft(-0.1, 0.1) == 0.0
    assert math.isclose(oracle.soft(0.35, 0.1), 0.25)
    assert math.isclose(oracle.soft(-0.35, 0.1), -0.25)
    assert oracle.soft(2.0, 0.0) == 2.0


def test_shrink_update_by_hand():
    # X = 0: W X = 0, t = b, d = soft(b) on bands 1..8 and d = b on band 0,
    # b' = t - d, g = W^T(2d - t), ||W X - d|| = ||d||.
    n = 5
    rng = np.random.Generator(np.random.PCG64(4))
    b = rng.uniform(-1, 1, (9, n, n))
    tau = 0.3
    bn, g, r = oracle.shrink(np.zeros((n, n)), b, tau)
    d = np.sign(b) * np.maximum(np.abs(b) - tau, 0.0)
    d[0] = b[0]
    assert np.allclose(bn, b - d, atol=1e-15)
    assert np.allclose(g, oracle.framelet_adjoint(2 * d - b), atol=1e-14)
    assert math.isclose(r, np.linalg.norm(d), rel_tol=1e-13)
    assert np.all(bn[0] == 0.0)
