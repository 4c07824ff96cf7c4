"""Serving form: continuous batching under an HBM budget (pytest -m gpu).

The main check is the one the serving contract asks for: every request's
image is the same when it is served in a mix of concurrent requests of
different sizes, view counts and precisions as when it is solved alone."""
import dataclasses
import time

import numpy as np
import pytest

from paper_1310_1434_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1310_1434_gb300 import air

GB = 1 << 30


def mix():
    ws = [inputs._wl("s0", 64, 2.0, 48, 96, 11, 5, 2, 2e4, n_outer=3, n_cg=3),
          inputs._wl("s1", 128, 1.0, 90, 192, 12, 6, 2, 2e4, n_outer=4, n_cg=2),
          inputs._wl("s2", 96, 1.5, 60, 150, 13, 5, 2, 2e4, n_outer=2, n_cg=4),
          inputs._wl("s3", 48, 2.5, 30, 70, 14, 4, 1, 2e4, n_outer=5, n_cg=2)]
    ws.append(dataclasses.replace(ws[1], name="s1_tc", geom=dataclasses.replace(ws[1].geom, precision=1)))
    return ws


def alone(w, Y):
    plan = air.Plan(w.geom)
    Xd = torch.empty(w.geom.n ** 2, device="cuda")
    air.air_solve(plan, torch.as_tensor(Y, device="cuda"), w.lam, w.mu, w.n_outer, w.n_cg, Xd)
    torch.cuda.synchronize()
    return Xd.cpu().numpy()


def oracle_solve(w, Y):
    import oracle
    og = oracle.Geometry(**{k: getattr(w.geom, k) for k in oracle.Geometry.__dataclass_fields__})
    return oracle.solve(og, Y.astype(np.float64), w.lam, w.mu, w.n_outer, w.n_cg).ravel()


def test_results_alone_equal_results_in_the_mix():
    ws = mix()
    Ys = [inputs.make_case(w)[2].astype(np.float32).ravel() for w in ws]
    srv = air.Server(8 * GB, max_slots=16)
    ids = [srv.submit(w.geom, Y, w.lam, w.mu, w.n_outer, w.n_cg) for w, Y in zip(ws, Ys)]
    # a second wave arrives while the first is on the GPU
    ids2 = [srv.submit(w.geom, Y, w.lam, w.mu, w.n_outer, w.n_cg) for w, Y in zip(ws[:2], Ys[:2])]
    res = [srv.wait(rid, ws[i].geom.n) for i, rid in enumerate(ids)]
    res2 = [srv.wait(rid, ws[i].geom.n) for i, rid in enumerate(ids2)]
    srv.close()
    for w, Y, X in zip(ws, Ys, res):
        ref = alone(w, Y)
        assert np.all(np.isfinite(X))
        assert np.linalg.norm(X - ref) <= 1e-4 * np.linalg.norm(ref), w.name
        # every served result of the mix, FP32 and split-BF16, against the
        # FP64 oracle at the final-image tolerance
        orc = oracle_solve(w, Y)
        assert np.linalg.norm(X - orc) <= 1e-4 * np.linalg.norm(orc), w.name
    for w, Y, X, X1 in zip(ws, Ys, res2, res):
        assert np.linalg.norm(X - X1) <= 1e-6 * np.linalg.norm(X1), w.name
        orc = oracle_solve(w, Y)
        assert np.linalg.norm(X - orc) <= 1e-4 * np.linalg.norm(orc), w.name


def test_overlap_and_timing_records():
    # long enough (20 x 8 iterations) that submitting all three takes far less
    # time than any one solve; the longest first
    ws = [dataclasses.replace(mix()[i], n_outer=20, n_cg=8) for i in (1, 2, 0)]
    Ys = [inputs.make_case(w)[2].astype(np.float32).ravel() for w in ws]
    srv = air.Server(8 * GB, max_slots=16)
    # warm the plan pool, so that admission below is a pool lookup, not a plan
    # build (which can outlast a small solve)
    for w, rid in [(w, srv.submit(w.geom, Y, w.lam, w.mu, w.n_outer, w.n_cg)) for w, Y in zip(ws, Ys)]:
        srv.wait(rid, w.geom.n)
    import gc
    gc.disable()       # no collector pause between the three submissions
    try:
        ids = [srv.submit(w.geom, Y, w.lam, w.mu, w.n_outer, w.n_cg) for w, Y in zip(ws, Ys)]
    finally:
        gc.enable()
    done = {}
    t_end = time.time() + 60
    while len(done) < len(ids) and time.time() < t_end:
        for i, rid in enumerate(ids):
            if rid not in done:
                try:
                    tm = srv.times(rid)
                except air.AirError:
                    tm = None
                if tm is not None:
                    done[rid] = tm
                    assert srv.poll(rid, ws[i].geom.n) is not None
        time.sleep(0.001)
    srv.close()
    assert len(done) == len(ids)
    for t in done.values():
        assert t[0] <= t[1] <= t[2]
    # all three were resident together: each was admitted before any finished
    admits = max(t[1] for t in done.values())
    firsts = min(t[2] for t in done.values())
    assert admits <= firsts, sorted(done.values())


def test_budget_admits_one_at_a_time_and_rejects_oversize():
    w = mix()[1]
    Y = inputs.make_case(w)[2].astype(np.float32).ravel()
    need = air.Plan(w.geom).nbytes
    srv = air.Server(int(need * 1.5), max_slots=8)
    ids = [srv.submit(w.geom, Y, w.lam, w.mu, w.n_outer, w.n_cg) for _ in range(3)]
    outs = [srv.wait(rid, w.geom.n) for rid in ids]
    for X in outs[1:]:
        assert np.array_equal(X, outs[0])
    big = inputs.Geometry(1024, 0.4, 800, 1476)
    with pytest.raises(air.AirError) as e:
        srv.submit(big, np.zeros(800 * 1476, np.float32), 1e-3, 1.0, 1, 1)
    assert e.value.status == air.AIR_ERR_BUDGET
    srv.close()
