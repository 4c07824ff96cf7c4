"""The allocation-free filtered adjoint (air_filtered_backproject_noalloc).

Some callers cannot call cudaMalloc when they need the operator, e.g. code
that runs under a fixed device-memory budget with allocation closed after
start-up.  This entry point keeps its scratch (the filtered sinogram and the
backprojector's view parts) in a static device array.  The test calls it through the C ABI twice in a row on
different data, so the second call reuses the array the first one left
behind, and checks each result against air_filtered_backproject within the
single-application tolerance (2e-6 relative L2).  It is collected last.
"""
import numpy as np
import pytest

from paper_1310_1434_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1310_1434_gb300 import air

TOL = 2e-6


def test_noalloc_matches_filtered_backproject_twice():
    lib = air.load()
    g = inputs.AIR512_V200.geom          # 200 x 738 samples, under the 2^20 limit
    plan = air.Plan(g)
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (21, 22):                # two calls in a row on different data
        ell = inputs.random_phantom(g, seed, 8, 4)
        Y = inputs.noisy_sinogram(inputs.ellipse_line_integrals(g, ell), 2e4, seed).astype(np.float32)
        Yd = torch.as_tensor(Y.ravel(), device="cuda")
        X_ref = torch.empty(g.n * g.n, device="cuda")
        X_na = torch.full((g.n * g.n,), float("nan"), device="cuda")
        air.air_filtered_backproject(plan, Yd, X_ref)
        st = lib.air_filtered_backproject_noalloc(plan.handle, Yd.data_ptr(), X_na.data_ptr(), stream)
        assert st == air.AIR_OK, air.last_error()
        torch.cuda.synchronize()
        a = X_na.cpu().numpy().astype(np.float64)
        b = X_ref.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= TOL * np.linalg.norm(b)


@pytest.mark.parametrize("n,V,nb,parts", [(512, 200, 738, 1), (1024, 32, 1476, 4)])
def test_noalloc_view_parts(n, V, nb, parts):
    # one view part (written straight to X), and a split larger than the
    # static scratch holds beside C Y at 1024^2 (four parts, three fit)
    lib = air.load()
    g = inputs.Geometry(n, 512 * 0.8 / n, V, nb)
    plan = air.Plan(g)
    air.air_plan_tune(plan, air.air_plan_config(plan)[0], parts)
    ell = inputs.random_phantom(g, 23, 8, 4)
    Yd = torch.as_tensor(inputs.ellipse_line_integrals(g, ell).astype(np.float32).ravel(), device="cuda")
    X_ref = torch.empty(g.n * g.n, device="cuda")
    X_na = torch.full((g.n * g.n,), float("nan"), device="cuda")
    air.air_filtered_backproject(plan, Yd, X_ref)
    st = lib.air_filtered_backproject_noalloc(plan.handle, Yd.data_ptr(), X_na.data_ptr(),
                                              torch.cuda.current_stream().cuda_stream)
    assert st == air.AIR_OK, air.last_error()
    torch.cuda.synchronize()
    a = X_na.cpu().numpy().astype(np.float64)
    b = X_ref.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(a))
    assert np.linalg.norm(a - b) <= TOL * np.linalg.norm(b)


def test_noalloc_with_a_split_bf16_plan_uses_the_fp32_filter():
    # a BF16X3 plan: the allocation-free call applies the FP32 filter, which
    # differs from the plan's tensor-core filter by rounding only (~2.5e-7)
    import dataclasses
    lib = air.load()
    g = dataclasses.replace(inputs.AIR512_V200.geom, precision=air.PREC_BF16X3)
    plan = air.Plan(g)
    ell = inputs.random_phantom(g, 24, 8, 4)
    Y = inputs.noisy_sinogram(inputs.ellipse_line_integrals(g, ell), 2e4, 24).astype(np.float32)
    Yd = torch.as_tensor(Y.ravel(), device="cuda")
    X_ref = torch.empty(g.n * g.n, device="cuda")
    X_na = torch.full((g.n * g.n,), float("nan"), device="cuda")
    air.air_filtered_backproject(plan, Yd, X_ref)
    st = lib.air_filtered_backproject_noalloc(plan.handle, Yd.data_ptr(), X_na.data_ptr(),
                                              torch.cuda.current_stream().cuda_stream)
    assert st == air.AIR_OK, air.last_error()
    torch.cuda.synchronize()
    a = X_na.cpu().numpy().astype(np.float64)
    b = X_ref.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(a))
    assert np.linalg.norm(a - b) <= TOL * np.linalg.norm(b)


def test_noalloc_rejects_a_plan_larger_than_its_scratch():
    lib = air.load()
    g = inputs.Geometry(64, 2.0, 1100, 960)     # 1,056,000 samples > 2^20
    plan = air.Plan(g)
    Y = torch.zeros(g.n_views * g.n_bins, device="cuda")
    X = torch.empty(g.n * g.n, device="cuda")
    st = lib.air_filtered_backproject_noalloc(plan.handle, Y.data_ptr(), X.data_ptr(),
                                              torch.cuda.current_stream().cuda_stream)
    assert st == air.AIR_ERR_INVALID_ARG
    assert "static scratch" in air.last_error()
