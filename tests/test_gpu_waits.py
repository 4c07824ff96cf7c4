"""Bounded device-side waits give up, report AIR_ERR_TIMEOUT and leave the
plans usable (pytest -m gpu).

Every spin-wait in the library's kernels has a poll budget.  These tests set
that budget to zero with air_set_wait_budget, so that the persistent batch
kernel's grid barrier and the tensor-core filter's wait for its first operand
stage give up at once, and check that the calls report AIR_ERR_TIMEOUT and
that the same plans then solve correctly with the default budget.  No kernel
is made to hang: a wait with a zero budget returns without polling, and a
tensor-core CTA that gives up still drains its own copies (default budget)
before it exits.
"""
import dataclasses

import numpy as np
import pytest

from paper_1310_1434_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1310_1434_gb300 import air

DEV = "cuda:0"


def cases():
    return [inputs._wl("w0", 48, 1.7, 40, 70, 3, 5, 2, 1e5, n_outer=3, n_cg=3),
            inputs._wl("w1", 64, 1.2, 33, 96, 4, 5, 2, 1e5, n_outer=2, n_cg=4)]


def solve_alone(w, plan, Y):
    x = torch.empty(w.geom.n ** 2, device=DEV)
    air.air_solve(plan, Y, w.lam, w.mu, w.n_outer, w.n_cg, x)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.float64)


def batch_args(ws):
    return [w.lam for w in ws], [w.mu for w in ws], [w.n_outer for w in ws], [w.n_cg for w in ws]


def test_grid_barrier_timeout_is_reported_and_the_batch_recovers():
    ws = cases()
    Ys = [torch.as_tensor(inputs.make_case(w)[2].astype(np.float32).ravel(), device=DEV) for w in ws]
    plans = [air.Plan(w.geom) for w in ws]
    Xs = [torch.empty(w.geom.n ** 2, device=DEV) for w in ws]
    air.air_set_wait_budget(0)
    try:
        with pytest.raises(air.AirError) as e:
            air.air_solve_batch_persistent(plans, Ys, *batch_args(ws), Xs)
        assert e.value.status == air.AIR_ERR_TIMEOUT
    finally:
        air.air_set_wait_budget(-1)
    # the same plans, and the same captured graph, with the default budget
    for x in Xs:
        x.fill_(float("nan"))
    air.air_solve_batch_persistent(plans, Ys, *batch_args(ws), Xs)
    for w, p, Y, x in zip(ws, plans, Ys, Xs):
        a, b = x.cpu().numpy().astype(np.float64), solve_alone(w, p, Y)
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b), w.name


def test_tensor_core_wait_timeout_is_reported_cleared_and_recovered():
    g = inputs.Geometry(96, 1.2, 150, 200)          # 2 view tiles, 2 K chunks per parity
    plan = air.Plan(dataclasses.replace(g, precision=air.PREC_BF16X3))
    plan32 = air.Plan(g)
    Y = torch.as_tensor(inputs.random_sinogram(g.n_views, g.n_bins, 5).astype(np.float32).ravel(), device=DEV)
    Z = torch.empty_like(Y)
    air.air_set_wait_budget(0)
    try:
        air.air_filter(plan, Y, Z)
        with pytest.raises(air.AirError) as e:
            air.air_plan_status(plan)
        assert e.value.status == air.AIR_ERR_TIMEOUT
    finally:
        air.air_set_wait_budget(-1)
    air.air_plan_status(plan)                        # reading the timeout cleared it
    Z.fill_(float("nan"))
    air.air_filter(plan, Y, Z)
    air.air_plan_status(plan)
    Zr = torch.empty_like(Y)
    air.air_filter(plan32, Y, Zr)
    torch.cuda.synchronize()
    a, b = Z.cpu().numpy().astype(np.float64), Zr.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(a))
    assert np.linalg.norm(a - b) <= 2e-6 * np.linalg.norm(b)


def test_tensor_core_timeout_inside_a_grouped_batch():
    ws = cases()
    geoms = [dataclasses.replace(w.geom, precision=air.PREC_BF16X3) for w in ws]
    Ys = [torch.as_tensor(inputs.make_case(w)[2].astype(np.float32).ravel(), device=DEV) for w in ws]
    plans = [air.Plan(gg) for gg in geoms]
    Xs = [torch.empty(w.geom.n ** 2, device=DEV) for w in ws]
    air.air_set_wait_budget(0)
    try:
        with pytest.raises(air.AirError) as e:
            air.air_solve_batch(plans, Ys, *batch_args(ws), Xs)
        assert e.value.status == air.AIR_ERR_TIMEOUT
    finally:
        air.air_set_wait_budget(-1)
    for p in plans:
        air.air_plan_status(p)                       # the batch call read (and so cleared) every status
    air.air_solve_batch(plans, Ys, *batch_args(ws), Xs)
    for w, p, Y, x in zip(ws, plans, Ys, Xs):
        a, b = x.cpu().numpy().astype(np.float64), solve_alone(w, p, Y)
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b), w.name
