"""Precision form: the ramp filter on tcgen05 tensor cores in split BF16 (3
pieces per operand, 6 products, FP32 accumulation) plus an FP32 near band,
against the FP64 oracle (pytest -m gpu).  Same bounds as the FP32 path: a
single C or A'^T application within 2e-6 relative L2, a full reconstruction
within 1e-4."""
import dataclasses
import os

import numpy as np
import pytest

import oracle
from paper_1310_1434_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1310_1434_gb300 import air

DEV = "cuda:0"


def tc(g):
    return dataclasses.replace(g, precision=1)


def ogeom(g):
    return oracle.Geometry(**{k: getattr(g, k) for k in oracle.Geometry.__dataclass_fields__})


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def noisy(g, seed):
    ell = inputs.random_phantom(g, seed, 8, 4)
    return inputs.noisy_sinogram(inputs.ellipse_line_integrals(g, ell), 2e4, seed).astype(np.float32)


# sizes: fewer views than one 128-row MMA tile, bins below the 64-lag near
# band, ragged bins (738 -> 768 padded), and the full 800-view slice
CASES = [inputs.Geometry(32, 2.0, 13, 50), inputs.Geometry(64, 1.5, 37, 130),
         inputs.Geometry(96, 1.0, 130, 200), inputs.AIR512_V200.geom, inputs.AIR512_V800.geom]


@pytest.mark.parametrize("g", CASES, ids=lambda g: f"{g.n}_v{g.n_views}_b{g.n_bins}")
def test_tc_filter_and_filtered_adjoint(g):
    Y = noisy(g, 3)
    plan = air.Plan(tc(g))
    Yd = torch.as_tensor(Y.ravel(), device=DEV)
    Zd = torch.empty_like(Yd)
    air.air_filter(plan, Yd, Zd)
    Xd = torch.empty(g.n * g.n, device=DEV)
    air.air_filtered_backproject(plan, Yd, Xd)
    air.air_plan_status(plan)
    og = ogeom(g)
    Y64 = Y.astype(np.float64)
    assert rel(Zd.cpu().numpy(), oracle.filter(og, Y64).ravel()) <= 2e-6
    assert rel(Xd.cpu().numpy(), oracle.filtered_backproject(og, Y64).ravel()) <= 2e-6


def test_tc_full_size_solve_matches_stored_oracle():
    w = inputs.AIR512_V800
    ref = np.load(os.path.join(os.path.dirname(__file__), "golden", f"{w.name}_oracle.npz"))
    Y = inputs.make_case(w)[2].astype(np.float32)
    plan = air.Plan(tc(w.geom))
    Xd = torch.empty(w.geom.n ** 2, device=DEV)
    air.air_solve(plan, torch.as_tensor(Y.ravel(), device=DEV), w.lam, w.mu, w.n_outer, w.n_cg, Xd)
    air.air_plan_status(plan)
    assert rel(Xd.cpu().numpy(), ref["X"].astype(np.float64).ravel()) <= 1e-4


def test_tc_host_solve_small():
    w = inputs._wl("tc48", 48, 1.7, 40, 70, 9, 5, 2, 1e5, n_outer=4, n_cg=3)
    Y = inputs.make_case(w)[2].astype(np.float32)
    plan = air.Plan(tc(w.geom))
    X = np.zeros(w.geom.n ** 2, np.float32)
    air.air_solve_host(plan, np.ascontiguousarray(Y.ravel()), w.lam, w.mu, w.n_outer, w.n_cg, X)
    Xo = oracle.solve(ogeom(w.geom), Y.astype(np.float64), w.lam, w.mu, w.n_outer, w.n_cg)
    assert rel(X, Xo.ravel()) <= 1e-4
