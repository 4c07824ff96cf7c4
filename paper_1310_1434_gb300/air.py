"""Thin ctypes binding of the AIR C ABI (include/air.h).

Argument marshalling only: every step of the reconstruction runs in the CUDA
kernels of ``libair.so``.  Functions keep the C names; array arguments are
torch CUDA tensors (float32, contiguous) or raw device pointers (int), and the
stream defaults to torch's current stream.  A missing library raises -- there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from . import build as _build

AIR_OK = 0
AIR_ERR_INVALID_ARG = -1
AIR_ERR_OOM = -2
AIR_ERR_CUDA = -3
AIR_ERR_TIMEOUT = -4
AIR_ERR_BUDGET = -5
AIR_ERR_NOT_READY = -6
AIR_ERR_INTERNAL = -7
FILTER_NONE, FILTER_RAMLAK = 0, 1
PREC_FP32, PREC_BF16X3 = 0, 1

# every symbol include/air.h declares
EXPORTS = ["air_last_error", "air_plan_create", "air_plan_destroy", "air_plan_bytes", "air_plan_status",
           "air_set_wait_budget", "air_plan_tune", "air_plan_config",
           "air_project",
           "air_filter", "air_backproject", "air_filtered_backproject", "air_filtered_backproject_noalloc",
           "air_framelet", "air_shrink",
           "air_solve", "air_solve_l2", "air_solve_fbs", "air_fbp", "air_solve_host",
           "air_solve_batch", "air_solve_batch_host", "air_solve_batch_persistent", "air_batch_graph_info",
           "air_server_create", "air_server_submit", "air_server_poll", "air_server_wait", "air_server_times",
           "air_server_destroy"]


class AirError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        super().__init__(f"{fn} failed with status {status}: {msg}")
        self.status = status


class air_geometry(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("pixel_mm", ctypes.c_double), ("n_views", ctypes.c_int32),
                ("n_bins", ctypes.c_int32), ("dso_mm", ctypes.c_double), ("dsd_mm", ctypes.c_double),
                ("dgamma", ctypes.c_double), ("beta0", ctypes.c_double), ("arc", ctypes.c_double),
                ("filter", ctypes.c_int32), ("precision", ctypes.c_int32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libair.so (building it first if asked).  Raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"AIR CUDA library not built ({path}); run __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, f32, u64 = ctypes.c_int, ctypes.c_float, ctypes.c_uint64
    g = ctypes.POINTER(air_geometry)
    sig = {
        "air_last_error": (ctypes.c_char_p, []),
        "air_plan_create": (i32, [g, ctypes.POINTER(P)]),
        "air_plan_destroy": (i32, [P]),
        "air_plan_bytes": (ctypes.c_size_t, [P]),
        "air_plan_status": (i32, [P]),
        "air_set_wait_budget": (i32, [ctypes.c_int64]),
        "air_plan_tune": (i32, [P, i32, i32]),
        "air_plan_config": (i32, [P, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "air_project": (i32, [P, P, P, P]),
        "air_filter": (i32, [P, P, P, P]),
        "air_backproject": (i32, [P, P, P, P]),
        "air_filtered_backproject": (i32, [P, P, P, P]),
        "air_filtered_backproject_noalloc": (i32, [P, P, P, P]),
        "air_framelet": (i32, [P, P, P, i32, P]),
        "air_shrink": (i32, [P, P, P, P, f32, P, P]),
        "air_solve": (i32, [P, P, f32, f32, i32, i32, P, P, P]),
        "air_solve_host": (i32, [P, P, f32, f32, i32, i32, P, P]),
        "air_solve_l2": (i32, [P, P, f32, i32, P, P]),
        "air_fbp": (i32, [P, P, P, P]),
        "air_solve_fbs": (i32, [P, P, f32, f32, i32, P, P]),
        "air_solve_batch": (i32, [i32, P, P, P, P, P, P, P, P]),
        "air_solve_batch_persistent": (i32, [i32, P, P, P, P, P, P, P, P]),
        "air_batch_graph_info": (i32, [ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_int64)]),
        "air_solve_batch_host": (i32, [i32, P, P, P, P, P, P, P, P]),
        "air_server_create": (i32, [ctypes.c_size_t, i32, ctypes.POINTER(P)]),
        "air_server_submit": (i32, [P, g, P, f32, f32, i32, i32, ctypes.POINTER(u64)]),
        "air_server_poll": (i32, [P, u64, P]),
        "air_server_wait": (i32, [P, u64, P]),
        "air_server_times": (i32, [P, u64, P]),
        "air_server_destroy": (i32, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return load().air_last_error().decode()


def _check(status: int, fn: str):
    if status != AIR_OK:
        raise AirError(status, fn, last_error())


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, int):
        return a
    import torch
    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if hasattr(a, "ctypes"):           # numpy array (host buffers)
        return a.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(a)}")


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


@dataclass
class Geometry:
    n: int
    pixel_mm: float
    n_views: int
    n_bins: int
    dso_mm: float = 850.0
    dsd_mm: float = 1450.0
    dgamma: float = 0.0
    beta0: float = 0.0
    arc: float = 6.283185307179586
    filter: int = FILTER_RAMLAK
    precision: int = PREC_FP32

    def c(self) -> air_geometry:
        return air_geometry(self.n, self.pixel_mm, self.n_views, self.n_bins, self.dso_mm, self.dsd_mm,
                            self.dgamma, self.beta0, self.arc, self.filter, self.precision)

    @classmethod
    def of(cls, g) -> "Geometry":
        return cls(**{k: getattr(g, k) for k in cls.__dataclass_fields__})


class Plan:
    """Owns an air_plan (geometry tables + workspace on the current device)."""

    def __init__(self, geom):
        self.geom = Geometry.of(geom)
        self._g = self.geom.c()
        h = ctypes.c_void_p()
        _check(load().air_plan_create(ctypes.byref(self._g), ctypes.byref(h)), "air_plan_create")
        self.handle = h.value

    def close(self):
        if getattr(self, "handle", None):
            load().air_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nbytes(self) -> int:
        return load().air_plan_bytes(self.handle)


def air_plan_create(geom) -> Plan:
    return Plan(geom)


def air_plan_destroy(plan: Plan):
    plan.close()


def air_plan_status(plan: Plan):
    _check(load().air_plan_status(plan.handle), "air_plan_status")


def air_set_wait_budget(polls: int):
    """Poll budget of the kernels' bounded waits on the current device (< 0: the default)."""
    _check(load().air_set_wait_budget(int(polls)), "air_set_wait_budget")


def air_plan_tune(plan: Plan, fwd_views_per_block: int, bwd_view_parts: int):
    _check(load().air_plan_tune(plan.handle, int(fwd_views_per_block), int(bwd_view_parts)), "air_plan_tune")


def air_plan_config(plan: Plan):
    """(views per projector block, backprojector view parts, largest allowed parts)."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().air_plan_config(plan.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "air_plan_config")
    return a.value, b.value, c.value


def air_project(plan: Plan, X, Y, stream=None):
    _check(load().air_project(plan.handle, _ptr(X), _ptr(Y), _stream(stream)), "air_project")


def air_filter(plan: Plan, Y, Z, stream=None):
    _check(load().air_filter(plan.handle, _ptr(Y), _ptr(Z), _stream(stream)), "air_filter")


def air_backproject(plan: Plan, Y, X, stream=None):
    _check(load().air_backproject(plan.handle, _ptr(Y), _ptr(X), _stream(stream)), "air_backproject")


def air_filtered_backproject(plan: Plan, Y, X, stream=None):
    _check(load().air_filtered_backproject(plan.handle, _ptr(Y), _ptr(X), _stream(stream)),
           "air_filtered_backproject")


def air_filtered_backproject_noalloc(plan: Plan, Y, X, stream=None):
    _check(load().air_filtered_backproject_noalloc(plan.handle, _ptr(Y), _ptr(X), _stream(stream)),
           "air_filtered_backproject_noalloc")


def air_framelet(plan: Plan, inp, out, adjoint: bool, stream=None):
    _check(load().air_framelet(plan.handle, _ptr(inp), _ptr(out), int(bool(adjoint)), _stream(stream)),
           "air_framelet")


def air_shrink(plan: Plan, X, b, g, thresh: float, resid=None, stream=None):
    _check(load().air_shrink(plan.handle, _ptr(X), _ptr(b), _ptr(g), float(thresh), _ptr(resid),
                             _stream(stream)), "air_shrink")


def air_solve(plan: Plan, Y, lam: float, mu: float, n_outer: int, n_cg: int, X, resid=None, stream=None):
    _check(load().air_solve(plan.handle, _ptr(Y), float(lam), float(mu), int(n_outer), int(n_cg), _ptr(X),
                            _ptr(resid), _stream(stream)), "air_solve")


def air_solve_l2(plan: Plan, Y, lam: float, n_cg: int, X, stream=None):
    _check(load().air_solve_l2(plan.handle, _ptr(Y), float(lam), int(n_cg), _ptr(X), _stream(stream)),
           "air_solve_l2")


def air_solve_fbs(plan: Plan, Y, lam: float, step: float, n_iter: int, X, stream=None):
    _check(load().air_solve_fbs(plan.handle, _ptr(Y), float(lam), float(step), int(n_iter), _ptr(X),
                                _stream(stream)), "air_solve_fbs")


def air_fbp(plan: Plan, Y, X, stream=None):
    _check(load().air_fbp(plan.handle, _ptr(Y), _ptr(X), _stream(stream)), "air_fbp")


def air_solve_host(plan: Plan, Y_host, lam: float, mu: float, n_outer: int, n_cg: int, X_host, stream=None):
    _check(load().air_solve_host(plan.handle, _ptr(Y_host), float(lam), float(mu), int(n_outer), int(n_cg),
                                 _ptr(X_host), _stream(stream)), "air_solve_host")


def _batch(fn, name, plans, Ys, lams, mus, n_outers, n_cgs, Xs, stream):
    n = len(plans)
    VP = ctypes.c_void_p * n
    _check(fn(n, ctypes.cast(VP(*[p.handle for p in plans]), ctypes.c_void_p),
              ctypes.cast(VP(*[_ptr(y) for y in Ys]), ctypes.c_void_p),
              ctypes.cast((ctypes.c_float * n)(*lams), ctypes.c_void_p),
              ctypes.cast((ctypes.c_float * n)(*mus), ctypes.c_void_p),
              ctypes.cast((ctypes.c_int * n)(*n_outers), ctypes.c_void_p),
              ctypes.cast((ctypes.c_int * n)(*n_cgs), ctypes.c_void_p),
              ctypes.cast(VP(*[_ptr(x) for x in Xs]), ctypes.c_void_p),
              _stream(stream)), name)


def air_solve_batch(plans, Ys, lams, mus, n_outers, n_cgs, Xs, stream=None):
    _batch(load().air_solve_batch, "air_solve_batch", plans, Ys, lams, mus, n_outers, n_cgs, Xs, stream)


def air_solve_batch_host(plans, Ys_host, lams, mus, n_outers, n_cgs, Xs_host, stream=None):
    """Ys_host / Xs_host: host arrays (numpy or CPU tensors, float32, contiguous;
    pinned memory makes the copies asynchronous)."""
    _batch(load().air_solve_batch_host, "air_solve_batch_host", plans, Ys_host, lams, mus, n_outers, n_cgs,
           Xs_host, stream)


def air_solve_batch_persistent(plans, Ys, lams, mus, n_outers, n_cgs, Xs, stream=None):
    _batch(load().air_solve_batch_persistent, "air_solve_batch_persistent", plans, Ys, lams, mus, n_outers,
           n_cgs, Xs, stream)


def air_batch_graph_info():
    """(chains, kernels per run) of the grouped batch graph in use."""
    c = ctypes.c_int(0)
    k = ctypes.c_int64(0)
    _check(load().air_batch_graph_info(ctypes.byref(c), ctypes.byref(k)), "air_batch_graph_info")
    return c.value, k.value


class Server:
    """Continuous-batching reconstruction server (air_server_*)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 64):
        h = ctypes.c_void_p()
        _check(load().air_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(h)),
               "air_server_create")
        self.handle = h.value
        self._side = {}    # request id -> image side, so result buffers are always n*n

    def submit(self, geom, Y_host, lam: float, mu: float, n_outer: int, n_cg: int) -> int:
        import numpy as np
        gg = Geometry.of(geom)
        g = gg.c()
        Y = np.ascontiguousarray(Y_host, dtype=np.float32)
        if Y.size != gg.n_views * gg.n_bins:
            raise ValueError(f"Y has {Y.size} values, the geometry {gg.n_views * gg.n_bins}")
        rid = ctypes.c_uint64()
        _check(load().air_server_submit(self.handle, ctypes.byref(g), Y.ctypes.data, float(lam), float(mu),
                                        int(n_outer), int(n_cg), ctypes.byref(rid)), "air_server_submit")
        self._side[rid.value] = gg.n
        return rid.value

    def _image(self, rid: int, n):
        import numpy as np
        side = self._side.get(rid)
        if side is None:
            raise KeyError(f"request {rid} was not submitted through this Server")
        if n is not None and int(n) != side:
            raise ValueError(f"request {rid} has a {side} x {side} image, not {n} x {n}")
        return np.empty(side * side, np.float32)

    def poll(self, rid: int, n: int = None):
        """The image (n*n float32) once finished, else None."""
        X = self._image(rid, n)
        st = load().air_server_poll(self.handle, rid, X.ctypes.data)
        if st == AIR_ERR_NOT_READY:
            return None
        _check(st, "air_server_poll")
        return X

    def wait(self, rid: int, n: int = None):
        X = self._image(rid, n)
        _check(load().air_server_wait(self.handle, rid, X.ctypes.data), "air_server_wait")
        return X

    def times(self, rid: int):
        t = (ctypes.c_double * 3)()
        _check(load().air_server_times(self.handle, rid, t), "air_server_times")
        return tuple(t)

    def close(self):
        if getattr(self, "handle", None):
            load().air_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
