"""L2-regularised AIR (Eq. 5) and forward-backward splitting AIR (Eq. 6 with
the framelet proximal step) through the C ABI against the FP64 oracle
(pytest -m gpu).  A reconstruction is within 1e-4 relative L2 of the oracle,
the tolerance of the final image of the split-Bregman path."""
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
TOL_SOLVE = 1e-4


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


def case(n, px, V, nb, seed, **kw):
    g = inputs.Geometry(n, px, V, nb, **kw)
    ell = inputs.random_phantom(g, seed, 6, 2)
    Y = f32(inputs.noisy_sinogram(inputs.ellipse_line_integrals(g, ell), 5e4, seed))
    return g, Y


def lipschitz(og, iters=30):
    """Largest eigenvalue of A'^T A = A^T C A (power iteration, oracle)."""
    x = np.random.Generator(np.random.PCG64(0)).standard_normal((og.n, og.n))
    lam = 0.0
    for _ in range(iters):
        y = oracle.filtered_backproject(og, oracle.project(og, x))
        lam = float(np.linalg.norm(y) / np.linalg.norm(x))
        x = y / np.linalg.norm(y)
    return lam


GEOMS = [dict(n=48, px=1.7, V=40, nb=70, seed=3),
         dict(n=77, px=1.3, V=31, nb=101, seed=4, beta0=0.7),           # ragged tiles
         dict(n=64, px=1.5, V=36, nb=90, seed=5, arc=3.6, beta0=0.2)]   # short scan


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
@pytest.mark.parametrize("gk", GEOMS, ids=["n48", "ragged77", "short64"])
def test_l2_air_matches_oracle(gk, prec):
    kw = dict(gk)
    g, Y = case(kw.pop("n"), kw.pop("px"), kw.pop("V"), kw.pop("nb"), kw.pop("seed"), **kw)
    og = ogeom(g)
    lam, n_cg = 0.05, 15
    ref = oracle.l2_solve(og, Y, lam, n_cg)
    plan = air.Plan(dataclasses.replace(g, precision=prec))
    X = torch.empty(g.n * g.n, device=DEV)
    air.air_solve_l2(plan, dev(Y), lam, n_cg, X)
    assert rel(host(X), ref.ravel()) <= TOL_SOLVE


def test_l2_ir_matches_oracle():
    """IR with the L2 regulariser: the same call with the filter off (C = I).
    A^T A is ill-conditioned without the filter, so lambda is a tenth of its
    largest eigenvalue: the condition number stays near 10 and 15 CG steps
    converge, where FP32 and FP64 runs of an unconverged CG would drift apart
    by about eps times the condition number."""
    g, Y = case(48, 1.7, 40, 70, 6, filter=0)
    og = ogeom(g)
    lam = 0.1 * lipschitz(og)
    ref = oracle.l2_solve(og, Y, lam, 15)
    plan = air.Plan(g)
    X = torch.empty(g.n * g.n, device=DEV)
    air.air_solve_l2(plan, dev(Y), lam, 15, X)
    assert rel(host(X), ref.ravel()) <= TOL_SOLVE


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
@pytest.mark.parametrize("gk", GEOMS, ids=["n48", "ragged77", "short64"])
def test_fbs_air_matches_oracle(gk, prec):
    kw = dict(gk)
    g, Y = case(kw.pop("n"), kw.pop("px"), kw.pop("V"), kw.pop("nb"), kw.pop("seed"), **kw)
    og = ogeom(g)
    step = 1.0 / lipschitz(og)
    c = oracle.framelet(oracle.filtered_backproject(og, Y))[1:]
    lam = 0.3 * float(np.abs(c).mean())    # threshold step*lam: a fair share of the coefficients of W X_half
    ref = oracle.fbs(og, Y, lam, step, 25)
    plan = air.Plan(dataclasses.replace(g, precision=prec))
    X = torch.empty(g.n * g.n, device=DEV)
    air.air_solve_fbs(plan, dev(Y), lam, step, 25, X)
    assert rel(host(X), ref.ravel()) <= TOL_SOLVE


def test_fbs_edge_cases():
    g, Y = case(48, 1.7, 40, 70, 7)
    og = ogeom(g)
    plan = air.Plan(g)
    X = torch.full((g.n * g.n,), float("nan"), device=DEV)
    air.air_solve_fbs(plan, dev(Y), 0.1, 0.5, 0, X)           # no iterations: X = 0
    assert np.all(host(X) == 0.0)
    air.air_solve_fbs(plan, dev(np.zeros_like(Y)), 0.1, 0.5, 5, X)   # zero data: X stays 0
    assert np.all(host(X) == 0.0)
    with pytest.raises(air.AirError):
        air.air_solve_fbs(plan, dev(Y), 0.1, 0.0, 5, X)       # step must be > 0
    with pytest.raises(air.AirError):
        air.air_solve_l2(plan, dev(Y), 0.0, 5, X)             # lambda must be > 0


# ------------------------------------------------------------- full size ----
@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_full_size_l2_and_fbs_match_oracle(prec):
    """A few iterations at 512^2 / 800 views / 738 bins (the oracle needs about
    a second per operator pair)."""
    w = inputs.AIR512_V800
    g = dataclasses.replace(w.geom, precision=prec)
    Y = f32(inputs.make_case(w)[2])
    og = ogeom(w.geom)
    plan = air.Plan(g)
    X = torch.empty(g.n * g.n, device=DEV)
    air.air_solve_l2(plan, dev(Y), 0.05, 3, X)
    assert rel(host(X), oracle.l2_solve(og, Y, 0.05, 3).ravel()) <= TOL_SOLVE
    air.air_solve_fbs(plan, dev(Y), 2e-3, 0.8, 2, X)
    assert rel(host(X), oracle.fbs(og, Y, 2e-3, 0.8, 2).ravel()) <= TOL_SOLVE


def test_full_size_fbs_one_step_infinite_threshold_is_lowpass_blur():
    """At any size: one step from 0 with a threshold above every coefficient
    is the periodic [1,4,6,4,1]/16 blur of step A'^T Y (checked against the
    library's own A'^T)."""
    w = inputs.AIR512_V800
    g = w.geom
    Y = f32(inputs.make_case(w)[2])
    plan = air.Plan(g)
    X = torch.empty(g.n * g.n, device=DEV)
    air.air_solve_fbs(plan, dev(Y), 1e30, 0.5, 1, X)
    B = torch.empty(g.n * g.n, device=DEV)
    air.air_filtered_backproject(plan, dev(Y), B)
    Xh = 0.5 * host(B).reshape(g.n, g.n)
    k = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0
    blur = sum(k[i] * np.roll(Xh, i - 2, axis=0) for i in range(5))
    blur = sum(k[i] * np.roll(blur, i - 2, axis=1) for i in range(5))
    assert rel(host(X).reshape(g.n, g.n), blur) <= 2e-6
