"""The C ABI library loads and exports what include/air.h declares, and the
host-side argument checks run without a GPU (no compute is launched)."""
import ctypes
import os
import re

import pytest

from paper_1310_1434_gb300 import air, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "air.h")


def declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^AIR_API[^(]*?\b(air_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return air.load()


def test_header_declares_the_binding_exports():
    assert declared() == sorted(air.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_invalid_geometry_rejected_on_host(lib):
    bad = [dict(n=0), dict(n=5000), dict(pixel_mm=0.0), dict(n_views=0), dict(n_bins=9000),
           dict(dso_mm=10.0), dict(dgamma=-1.0), dict(arc=0.0), dict(filter=7), dict(precision=3)]
    for kw in bad:
        g = air.Geometry(n=64, pixel_mm=1.0, n_views=10, n_bins=96)
        for k, v in kw.items():
            setattr(g, k, v)
        h = ctypes.c_void_p()
        st = lib.air_plan_create(ctypes.byref(g.c()), ctypes.byref(h))
        assert st == air.AIR_ERR_INVALID_ARG, kw
        assert h.value is None
        assert air.last_error()


def test_null_arguments_rejected_on_host(lib):
    h = ctypes.c_void_p()
    assert lib.air_plan_create(None, ctypes.byref(h)) == air.AIR_ERR_INVALID_ARG
    assert lib.air_project(None, None, None, None) == air.AIR_ERR_INVALID_ARG
    assert lib.air_solve(None, None, 0.0, 1.0, 1, 1, None, None, None) == air.AIR_ERR_INVALID_ARG
    assert lib.air_solve_batch(0, None, None, None, None, None, None, None, None) == air.AIR_ERR_INVALID_ARG
    assert lib.air_plan_destroy(None) == air.AIR_OK


def test_server_arguments_rejected_on_host(lib):
    h = ctypes.c_void_p()
    assert lib.air_server_create(0, 4, ctypes.byref(h)) == air.AIR_ERR_INVALID_ARG
    assert lib.air_server_create(1 << 30, 0, ctypes.byref(h)) == air.AIR_ERR_INVALID_ARG
    assert lib.air_server_create(1 << 30, 4, None) == air.AIR_ERR_INVALID_ARG
    assert lib.air_server_poll(None, 1, None) == air.AIR_ERR_INVALID_ARG
    assert lib.air_server_destroy(None) == air.AIR_OK
