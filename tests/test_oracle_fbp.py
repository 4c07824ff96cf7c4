"""Pins of the oracle's fan-beam FBP (the analytic reconstruction the paper
compares AIR with, Materials) against closed forms of analytic phantoms: exact
line integrals of disks (no discretised object) reconstruct to the disk's
density, mass and position."""
import math

import numpy as np
import pytest

import oracle
from paper_1310_1434_gb300 import inputs

N, PX, V, NB = 64, 2.0, 720, 257
# a short source distance (fan angles up to 0.47 rad, cos gamma down to 0.89) so
# that the pre-weight and the fan ramp's (gamma / sin gamma)^2 matter
DSO = 250.0


def geom():
    return inputs.Geometry(N, PX, V, NB, dso_mm=DSO, dsd_mm=2 * DSO)


def ogeom(g):
    return oracle.Geometry(**{k: getattr(g, k) for k in oracle.Geometry.__dataclass_fields__})


def disk(cx, cy, r, mu):
    return [inputs.Ellipse(cx, cy, r, r, 0.0, mu)]


def centres():
    c = (np.arange(N) + 0.5 - 0.5 * N) * PX
    return np.meshgrid(c, c)          # X[iy, ix], Y[iy, ix]


def test_taps_are_the_fan_ramp():
    """g(m alpha) = (1/2) (m alpha / sin m alpha)^2 h(m alpha) with the
    band-limited ramp h(0) = 1/(4 alpha^2), h(odd m) = -1/(pi m alpha)^2."""
    g = ogeom(geom())
    a = oracle.dgamma(g)
    t = oracle.fbp_taps(g)
    for m in (1, 3, 7, 31):
        h = -1.0 / (math.pi * m * a) ** 2
        assert t[m] == pytest.approx(0.5 * (m * a / math.sin(m * a)) ** 2 * h, rel=1e-12)
    assert t[0] == pytest.approx(0.5 / (4 * a * a), rel=1e-14)
    assert np.all(t[2::2] == 0.0)


def test_centred_disk_reconstructs_its_density():
    """Interior within 0.5 % of the density (mean within 0.1 %), and nothing
    beyond the rim: the scale (D, alpha, dbeta, 1/L^2) and the fan ramp."""
    g = geom()
    mu, r = 0.02, 40.0
    Y = inputs.ellipse_line_integrals(g, disk(0.0, 0.0, r, mu))
    f = oracle.fbp(ogeom(g), Y)
    X, Yc = centres()
    rad = np.hypot(X, Yc)
    inside = rad < r - 2 * PX
    outside = (rad > r + 3 * PX) & (rad < r + 10 * PX) & (rad < 0.48 * N * PX)
    assert abs(f[inside].mean() / mu - 1.0) < 1e-3
    assert np.abs(f[inside] / mu - 1.0).max() < 5e-3
    assert np.abs(f[outside]).max() < 8e-3 * mu


@pytest.mark.parametrize("cx, cy, r", [(45.0, 0.0, 12.0), (0.0, 55.0, 6.0), (30.0, 30.0, 15.0),
                                       (-35.0, 10.0, 20.0)])
def test_offcentre_disk_reconstructs_its_density(cx, cy, r):
    """Off-centre objects, seen at large fan angles, test the cos-gamma
    pre-weight and the 1/L^2 weight: every interior pixel within 0.5 %."""
    g = geom()
    mu = 0.02
    Y = inputs.ellipse_line_integrals(g, disk(cx, cy, r, mu))
    f = oracle.fbp(ogeom(g), Y)
    X, Yc = centres()
    inside = np.hypot(X - cx, Yc - cy) < r - 2 * PX
    assert np.abs(f[inside] / mu - 1.0).max() < 5e-3


@pytest.mark.parametrize("cx, cy", [(0.0, 0.0), (30.0, -12.0), (-8.0, 38.0)])
def test_small_disk_mass_and_position(cx, cy):
    """A small disk reconstructs where it is (centroid) with its mass (to the
    few per cent a pixel sum of a 4-pixel disk allows)."""
    g = geom()
    mu, r = 0.05, 8.0
    Y = inputs.ellipse_line_integrals(g, disk(cx, cy, r, mu))
    f = oracle.fbp(ogeom(g), Y)
    X, Yc = centres()
    near = np.hypot(X - cx, Yc - cy) < 4 * r
    mass = f[near].sum() * PX * PX
    assert abs(mass / (mu * math.pi * r * r) - 1.0) < 4e-2
    w = np.clip(f, 0, None) * near
    assert abs((w * X).sum() / w.sum() - cx) < 0.1 * PX
    assert abs((w * Yc).sum() / w.sum() - cy) < 0.1 * PX


def test_pixel_subset_matches_full_image():
    g = geom()
    Y = inputs.ellipse_line_integrals(g, disk(10.0, 5.0, 20.0, 0.02))
    full = oracle.fbp(ogeom(g), Y)
    iy, ix = np.array([0, 5, 33, 63]), np.array([7, 63, 32, 0])
    assert np.array_equal(oracle.fbp(ogeom(g), Y, (iy, ix)), full[iy, ix])


def test_filter_impulse_response_is_the_even_fan_ramp_at_the_impulse():
    """An impulse at bin j0 filters to alpha D cos(gamma_j0) g((j - j0) alpha):
    symmetric about j0, largest there, and zero at even offsets."""
    g = ogeom(geom())
    Y = np.zeros((V, NB))
    j0 = 100
    Y[3, j0] = 1.0
    Q = oracle.fbp_filter(g, Y)
    assert np.all(Q[:3] == 0.0) and np.all(Q[4:] == 0.0)
    q = Q[3]
    assert int(np.argmax(q)) == j0
    m = np.arange(1, 100)
    assert np.allclose(q[j0 + m], q[j0 - m], rtol=1e-12, atol=0)
    assert np.all(q[j0 + m[m % 2 == 0]] == 0.0)
    a = oracle.dgamma(g)
    assert q[j0] == pytest.approx(a * g.dso_mm * math.cos((j0 - 0.5 * (NB - 1)) * a) * oracle.fbp_taps(g)[0],
                                  rel=1e-12)
