"""FP64 CPU oracle for AIR (arXiv 1310.1434) -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is a plain, slow, double-precision
C implementation (``oracle/*.c``, built with gcc) of what the GPU library
computes, written from the paper's definitions and sharing no code with it:

* ``project`` / ``backproject``: the X-ray transform A of Eq. (1) by Siddon's
  method and its explicit transpose;
* ``filter`` / ``filtered_backproject``: the filtration C of Eq. (2) (FFT
  Ram-Lak, linear convolution) and A'^T = A^T C of Eq. (5);
* ``framelet`` / ``framelet_adjoint`` / ``shrink``: the tensor framelet W and
  the split-Bregman d/b update;
* ``cg`` / ``solve``: the CG-solved L2 step and the split-Bregman loop;
* ``l2_solve`` / ``fbs``: L2-regularised AIR (Eq. 5) and forward-backward
  splitting AIR (Eq. 6 plus the framelet proximal step), in numpy over the
  functions above;
* ``fbp``: the analytic reconstruction the paper compares against (FBP,
  Materials), the textbook equiangular fan-beam algorithm, in numpy.

Pins against the paper and the mathematics live in ``tests/test_oracle_*.py``.
Parity of the full-size configurations beyond those pins is "parity
unpinned": the oracle is then the reference by construction.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = ["siddon.c", "ramp.c", "framelet.c", "solver.c"]
_LIB_PATH = os.path.join(_HERE, "_build", "liborc.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math) into _build/."""
    srcs = [os.path.join(_HERE, s) for s in _SRC] + [os.path.join(_HERE, "orc.h")]
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
           "-fopenmp", "-fno-fast-math", "-ffp-contract=off", "-o", tmp] + \
          [os.path.join(_HERE, s) for s in _SRC] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Geom(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("pixel_mm", ctypes.c_double),
                ("n_views", ctypes.c_int), ("n_bins", ctypes.c_int),
                ("dso_mm", ctypes.c_double), ("dsd_mm", ctypes.c_double),
                ("dgamma", ctypes.c_double), ("beta0", ctypes.c_double),
                ("arc", ctypes.c_double), ("filter", ctypes.c_int)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d = ctypes.c_double
        g = P(_Geom)
        dp = P(d)
        sig = {
            "orc_dgamma": (d, [g]),
            "orc_ray": (None, [g, ctypes.c_int, ctypes.c_int, dp, dp]),
            "orc_ray_segments": (ctypes.c_int, [g, ctypes.c_int, ctypes.c_int,
                                                P(ctypes.c_int), dp, ctypes.c_int]),
            "orc_project_ray": (d, [g, dp, ctypes.c_int, ctypes.c_int]),
            "orc_project": (None, [g, dp, dp]),
            "orc_backproject": (None, [g, dp, dp]),
            "orc_ramp_tap": (d, [ctypes.c_int]),
            "orc_ramp_scale": (d, [g]),
            "orc_filter": (None, [g, dp, dp]),
            "orc_filtered_backproject": (None, [g, dp, dp]),
            "orc_framelet": (None, [ctypes.c_int, dp, dp]),
            "orc_framelet_adjoint": (None, [ctypes.c_int, dp, dp]),
            "orc_soft": (d, [d, d]),
            "orc_shrink": (d, [ctypes.c_int, dp, dp, dp, d]),
            "orc_cg": (None, [g, dp, d, ctypes.c_int, dp]),
            "orc_solve": (None, [g, dp, d, d, ctypes.c_int, ctypes.c_int, dp, dp]),
            "orc_threads": (ctypes.c_int, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


@dataclass
class Geometry:
    """Fan-beam geometry (mm, rad); mirrors the fields of the C struct."""
    n: int
    pixel_mm: float
    n_views: int
    n_bins: int
    dso_mm: float = 850.0
    dsd_mm: float = 1450.0
    dgamma: float = 0.0
    beta0: float = 0.0
    arc: float = 2.0 * np.pi
    filter: int = 1

    def _c(self) -> _Geom:
        return _Geom(self.n, self.pixel_mm, self.n_views, self.n_bins, self.dso_mm,
                     self.dsd_mm, self.dgamma, self.beta0, self.arc, self.filter)


def _geom(g) -> _Geom:
    if isinstance(g, _Geom):
        return g
    if isinstance(g, Geometry):
        return g._c()
    return Geometry(**{k: getattr(g, k) for k in Geometry.__dataclass_fields__})._c()


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def threads() -> int:
    return _load().orc_threads()


def dgamma(g) -> float:
    return _load().orc_dgamma(ctypes.byref(_geom(g)))


def ray(g, v: int, j: int):
    s = np.zeros(2)
    u = np.zeros(2)
    _load().orc_ray(ctypes.byref(_geom(g)), v, j, _dptr(s), _dptr(u))
    return s, u


def ray_segments(g, v: int, j: int):
    """(pixel indices, lengths) of ray (v, j), in the order Siddon visits them."""
    cg = _geom(g)
    cap = 4 * cg.n + 8
    pix = np.zeros(cap, dtype=np.int32)
    ln = np.zeros(cap)
    m = _load().orc_ray_segments(ctypes.byref(cg), v, j,
                                 pix.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(ln), cap)
    return pix[:m].copy(), ln[:m].copy()


def project_ray(g, X, v: int, j: int) -> float:
    X = _f64(X)
    return _load().orc_project_ray(ctypes.byref(_geom(g)), _dptr(X), v, j)


def project(g, X) -> np.ndarray:
    cg = _geom(g)
    X = _f64(X).reshape(-1)
    assert X.size == cg.n * cg.n
    Y = np.zeros((cg.n_views, cg.n_bins))
    _load().orc_project(ctypes.byref(cg), _dptr(X), _dptr(Y))
    return Y


def backproject(g, Y) -> np.ndarray:
    cg = _geom(g)
    Y = _f64(Y).reshape(-1)
    assert Y.size == cg.n_views * cg.n_bins
    X = np.zeros((cg.n, cg.n))
    _load().orc_backproject(ctypes.byref(cg), _dptr(Y), _dptr(X))
    return X


def ramp_tap(k: int) -> float:
    return _load().orc_ramp_tap(k)


def ramp_scale(g) -> float:
    return _load().orc_ramp_scale(ctypes.byref(_geom(g)))


def filter(g, Y) -> np.ndarray:  # noqa: A001 - the paper's name for C
    cg = _geom(g)
    Y = _f64(Y).reshape(-1)
    Z = np.zeros((cg.n_views, cg.n_bins))
    _load().orc_filter(ctypes.byref(cg), _dptr(Y), _dptr(Z))
    return Z


def filtered_backproject(g, Y) -> np.ndarray:
    cg = _geom(g)
    Y = _f64(Y).reshape(-1)
    X = np.zeros((cg.n, cg.n))
    _load().orc_filtered_backproject(ctypes.byref(cg), _dptr(Y), _dptr(X))
    return X


def framelet(X) -> np.ndarray:
    X = _f64(X)
    n = X.shape[0]
    c = np.zeros((9, n, n))
    _load().orc_framelet(n, _dptr(X), _dptr(c))
    return c


def framelet_adjoint(c) -> np.ndarray:
    c = _f64(c)
    n = c.shape[1]
    X = np.zeros((n, n))
    _load().orc_framelet_adjoint(n, _dptr(c), _dptr(X))
    return X


def soft(t: float, tau: float) -> float:
    return _load().orc_soft(t, tau)


def shrink(X, b, tau: float):
    """Returns (b_new, g, ||WX - d||_2); b is not modified."""
    X = _f64(X)
    n = X.shape[0]
    bn = _f64(b).copy()
    g = np.zeros((n, n))
    r = _load().orc_shrink(n, _dptr(X), _dptr(bn), _dptr(g), tau)
    return bn, g, r


def cg(g, rhs, mu: float, n_cg: int, X0=None) -> np.ndarray:
    cg_ = _geom(g)
    rhs = _f64(rhs)
    X = np.zeros((cg_.n, cg_.n)) if X0 is None else _f64(X0).copy()
    _load().orc_cg(ctypes.byref(cg_), _dptr(rhs), mu, n_cg, _dptr(X))
    return X


def solve(g, Y, lam: float, mu: float, n_outer: int, n_cg: int, return_resid=False):
    cg_ = _geom(g)
    Y = _f64(Y)
    X = np.zeros((cg_.n, cg_.n))
    r = np.zeros(max(n_outer, 1))
    _load().orc_solve(ctypes.byref(cg_), _dptr(Y), lam, mu, n_outer, n_cg, _dptr(X), _dptr(r))
    return (X, r[:n_outer]) if return_resid else X


def l2_solve(g, Y, lam: float, n_cg: int) -> np.ndarray:
    """L2-regularised AIR, Eq. (5): (A'^T A + lam I) X = A'^T Y with
    A'^T = A^T C, by n_cg conjugate-gradient steps from X = 0."""
    return cg(g, filtered_backproject(g, Y), lam, n_cg)


def fbs(g, Y, lam: float, step: float, n_iter: int) -> np.ndarray:
    """Forward-backward splitting AIR (Methods, Eq. 6) for
    min 1/2 ||P(AX - Y)||^2 + lam ||W X||_1 from X = 0:
      X_half = X - step A'^T (A X - Y)                      (Eq. 6)
      X      = W^T S(W X_half),  S = soft threshold step * lam on the
               high-pass bands 1..8, band 0 unchanged (the proximal step with
               the tight frame W, W^T W = I)."""
    cg_ = _geom(g)
    Y = _f64(Y).reshape(cg_.n_views, cg_.n_bins)
    X = np.zeros((cg_.n, cg_.n))
    t = step * lam
    for _ in range(n_iter):
        Xh = X - step * filtered_backproject(g, project(g, X) - Y)
        c = framelet(Xh)
        c[1:] = np.sign(c[1:]) * np.maximum(np.abs(c[1:]) - t, 0.0)
        X = framelet_adjoint(c)
    return X


def fbp_taps(g) -> np.ndarray:
    """The equiangular fan-beam ramp g(m alpha), m = 0 .. n_bins-1 (alpha the
    fan pitch): 1/(8 alpha^2) at 0, 0 at even m, -1/(2 pi^2 sin^2(m alpha)) at
    odd m -- the band-limited ramp h(m alpha) times (1/2)(m alpha/sin m alpha)^2."""
    cg_ = _geom(g)
    a = dgamma(g)
    m = np.arange(cg_.n_bins, dtype=np.float64)
    t = np.zeros(cg_.n_bins)
    t[0] = 1.0 / (8.0 * a * a)
    odd = m % 2 == 1
    t[odd] = -1.0 / (2.0 * np.pi ** 2 * np.sin(m[odd] * a) ** 2)
    return t


def fbp_filter(g, Y) -> np.ndarray:
    """The filtering half of fan-beam FBP, per view:
    Q(j) = alpha sum_k D cos(gamma_k) Y(k) g((j - k) alpha)."""
    cg_ = _geom(g)
    V, nb = cg_.n_views, cg_.n_bins
    Y = _f64(Y).reshape(V, nb)
    a = dgamma(g)
    gam = (np.arange(nb) - 0.5 * (nb - 1)) * a
    taps = fbp_taps(g)
    full = np.concatenate([taps[:0:-1], taps])          # g(m), m = -(nb-1) .. nb-1
    Q = np.empty((V, nb))
    for v in range(V):
        Q[v] = a * np.convolve(cg_.dso_mm * np.cos(gam) * Y[v], full)[nb - 1:2 * nb - 1]
    return Q


def fbp(g, Y, pixels=None) -> np.ndarray:
    """Equiangular fan-beam filtered backprojection of a full 2 pi scan:
      R'_v(j) = D cos(gamma_j) Y_v(j)                       (pre-weight)
      Q_v(j)  = alpha sum_k R'_v(k) g((j - k) alpha)         (fan ramp, fbp_taps)
      f(x, y) = dbeta sum_v Q_v(gamma'(x, y)) / L_v(x, y)^2  (weighted backprojection)
    with D the source-isocentre distance, gamma' the fan angle of the pixel
    centre seen from source v, L its distance from the source, dbeta = 2 pi/V,
    and Q linearly interpolated between bins (zero beyond the detector).
    ``pixels``: optional (iy, ix) index arrays; returns f at those pixels only."""
    cg_ = _geom(g)
    n, V, nb = cg_.n, cg_.n_views, cg_.n_bins
    Qall = fbp_filter(g, Y)
    a = dgamma(g)
    D = cg_.dso_mm
    jm = 0.5 * (nb - 1)
    if pixels is None:
        iy, ix = np.mgrid[0:n, 0:n]
    else:
        iy, ix = np.asarray(pixels[0]), np.asarray(pixels[1])
    x = (ix + 0.5 - 0.5 * n) * cg_.pixel_mm
    y = (iy + 0.5 - 0.5 * n) * cg_.pixel_mm
    f = np.zeros(x.shape)
    for v in range(V):
        beta = cg_.beta0 + cg_.arc * v / V
        Q = Qall[v]
        Sx, Sy = D * np.cos(beta), D * np.sin(beta)
        cx, cy = -np.cos(beta), -np.sin(beta)
        ux, uy = x - Sx, y - Sy
        gp = np.arctan2(cx * uy - cy * ux, cx * ux + cy * uy)
        t = gp / a + jm
        j0 = np.floor(t).astype(np.int64)
        w = t - j0
        Qz = np.concatenate([[0.0], Q, [0.0]])           # zero beyond the detector
        q0 = Qz[np.clip(j0, -1, nb) + 1]
        q1 = Qz[np.clip(j0 + 1, -1, nb) + 1]
        f += ((1.0 - w) * q0 + w * q1) / (ux * ux + uy * uy)
    return f * (cg_.arc / V)
