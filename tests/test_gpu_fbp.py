"""Fan-beam FBP (the paper's analytic comparison reconstruction) through the C
ABI against the FP64 oracle (pytest -m gpu).

Tolerance (derived from the arithmetic; the problem statement fixes none for
FBP): the GPU sums V terms per pixel in FP32, a random-walk error of about
sqrt(V) 2^-24 = 1.7e-6 relative at V = 800, and evaluates the fan angle in
FP32 from source-relative products (IEEE division, the bin fraction as an FMA
residual), which moves the interpolation point by at most ~2e-5 bins; the
image-wide relative L2 error is then below 5e-6 (measured 2.3e-6 at
512^2/800, 3.5e-7 to 5.6e-7 on the small cases).
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1310_1434_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1310_1434_gb300 import air

DEV = "cuda:0"
TOL_FBP = 5e-6


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def ogeom(g):
    return oracle.Geometry(**{k: getattr(g, k) for k in oracle.Geometry.__dataclass_fields__})


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=DEV)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


CASES = [dict(n=48, px=1.7, V=60, nb=70, seed=3),
         dict(n=77, px=1.3, V=90, nb=101, seed=4, beta0=0.7),                      # ragged tiles
         dict(n=64, px=2.0, V=120, nb=129, seed=5, dso_mm=250.0, dsd_mm=500.0)]    # fan angles to 0.47 rad


@pytest.mark.parametrize("ck", CASES, ids=["n48", "ragged77", "wide_fan"])
def test_fbp_matches_oracle(ck):
    kw = dict(ck)
    n, px, V, nb, seed = (kw.pop(k) for k in ("n", "px", "V", "nb", "seed"))
    g = inputs.Geometry(n, px, V, nb, **kw)
    ell = inputs.random_phantom(g, seed, 6, 2)
    Y = f32(inputs.noisy_sinogram(inputs.ellipse_line_integrals(g, ell), 5e4, seed))
    ref = oracle.fbp(ogeom(g), Y)
    plan = air.Plan(g)
    X = torch.empty(n * n, device=DEV)
    air.air_fbp(plan, dev(Y), X)
    assert rel(host(X), ref.ravel()) <= TOL_FBP


def test_fbp_is_linear_and_rejects_short_scans():
    g = inputs.Geometry(48, 1.7, 60, 70)
    rng = np.random.Generator(np.random.PCG64(8))
    Y1, Y2 = rng.standard_normal((2, 60 * 70)).astype(np.float32)
    plan = air.Plan(g)
    X1, X2, X3 = (torch.empty(48 * 48, device=DEV) for _ in range(3))
    air.air_fbp(plan, dev(Y1), X1)
    air.air_fbp(plan, dev(Y2), X2)
    air.air_fbp(plan, dev(Y1 + Y2), X3)
    a, b = host(X1) + host(X2), host(X3)
    assert rel(b, a) <= 1e-6
    Z = torch.zeros(60 * 70, device=DEV)
    air.air_fbp(plan, Z, X1)
    assert np.all(host(X1) == 0.0)
    short = air.Plan(dataclasses.replace(g, arc=3.5))
    with pytest.raises(air.AirError):
        air.air_fbp(short, dev(Y1), X1)


def test_full_size_fbp_matches_oracle_on_sampled_pixels():
    """512^2 / 800 views / 738 bins: the oracle evaluates 3,000 sampled pixels."""
    w = inputs.AIR512_V800
    g = w.geom
    Y = f32(inputs.make_case(w)[2])
    plan = air.Plan(g)
    X = torch.empty(g.n * g.n, device=DEV)
    air.air_fbp(plan, dev(Y), X)
    rng = np.random.Generator(np.random.PCG64(9))
    iy, ix = rng.integers(0, g.n, 3000), rng.integers(0, g.n, 3000)
    ref = oracle.fbp(ogeom(g), Y, (iy, ix))
    got = host(X).reshape(g.n, g.n)[iy, ix]
    assert rel(got, ref) <= TOL_FBP
