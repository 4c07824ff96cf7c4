"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds none of the reconstruction's arithmetic.  It plays the
scanner: random ellipse phantoms, their exact fan-beam line integrals, Poisson
counting noise, and random images/sinograms for operator tests.  The paper's
data (TomoTherapy MVCT scans of a Siemens image-quality phantom, Materials
section: 528 bins, 800 or 200 views per rotation, 350 x 350 pixels of 1 mm) are
not available; these phantoms stand in for them with the same structure
(fan-beam, full rotation, full and 25 % view counts, low-contrast ellipses plus
small high-contrast disks).

The scanner geometry follows the same conventions as the library: view v at
beta = beta0 + arc*v/V with the source at dso*(cos beta, sin beta); bin j at
fan angle gamma_j = (j - (n_b-1)/2)*dgamma, the ray leaving the source at angle
beta + pi + gamma_j; dgamma = 0 selects the fan that covers the image's
circumscribed circle.  Everything here is float64 numpy; the random stream is
numpy's PCG64 seeded per configuration.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
import math

import numpy as np

MU_MAX = 0.02  # attenuation scale of the phantoms, 1/mm (water-like at MV energies)


@dataclass(frozen=True)
class Geometry:
    n: int                 # image side N
    pixel_mm: float        # pixel pitch
    n_views: int           # V
    n_bins: int            # detector bins
    dso_mm: float = 850.0
    dsd_mm: float = 1450.0
    dgamma: float = 0.0    # 0 = automatic
    beta0: float = 0.0
    arc: float = 2.0 * math.pi
    filter: int = 1        # 1 = Ram-Lak (AIR), 0 = identity (IR)
    precision: int = 0     # 0 = FP32 filter, 1 = split-BF16 tensor-core filter

    @property
    def fan_pitch(self) -> float:
        if self.dgamma > 0:
            return self.dgamma
        r = self.n * self.pixel_mm / math.sqrt(2.0)
        return 2.0 * math.asin(r / self.dso_mm) / self.n_bins


@dataclass(frozen=True)
class Workload:
    """One reconstruction problem: geometry, phantom recipe, solver settings."""
    name: str
    geom: Geometry
    seed: int
    n_ellipses: int
    n_disks: int
    photons: float
    lam: float
    mu: float
    n_outer: int
    n_cg: int


def _wl(name, n, px, V, nb, seed, ne, nd, I0, lam=3e-4, mu=1.0, n_outer=30, n_cg=8, **kw):
    return Workload(name, Geometry(n, px, V, nb, **kw), seed, ne, nd, I0, lam, mu, n_outer, n_cg)


# The paper-shaped workloads (fan geometry: source-isocentre 850 mm,
# source-detector 1450 mm).  Pixel pitches and bin counts not fixed by the
# configuration list follow a 1.44*N bin rule and a ~410 mm field of view.
AIR128 = _wl("air128_v90", 128, 1.0, 90, 192, 0, 6, 0, 1e5, 0.01, 1.0, 20, 5)
AIR512_V800 = _wl("air512_v800", 512, 0.8, 800, 738, 1, 10, 12, 2e4)
AIR512_V200 = _wl("air512_v200", 512, 0.8, 200, 738, 1, 10, 12, 2e4)
AIR512_V800_BF16X3 = replace(AIR512_V800, name="air512_v800_bf16x3",
                             geom=replace(AIR512_V800.geom, precision=1))

# Batch of 64 slices of uneven geometry, seeds 100..163, sizes cycling.
_BATCH_SHAPES = [(256, 1.6, 200, 384), (512, 0.8, 400, 738),
                 (512, 0.8, 800, 738), (768, 0.8 * 512 / 768, 800, 1024)]


def batch_workloads(count: int = 64, first_seed: int = 100, n_outer=30, n_cg=8):
    out = []
    for i in range(count):
        n, px, V, nb = _BATCH_SHAPES[i % len(_BATCH_SHAPES)]
        out.append(_wl(f"batch{i}_{n}_v{V}", n, px, V, nb, first_seed + i, 8, 4, 2e4,
                       n_outer=n_outer, n_cg=n_cg))
    return out


SERVE_SIZES = [(256, 1.6, 384), (512, 0.8, 738), (1024, 0.4, 1476)]
SERVE_VIEWS = [200, 400, 800]


def serving_trace(count: int = 2000, rate_hz: float = 200.0, seed: int = 7,
                  n_outer=30, n_cg=8):
    """Poisson arrivals: list of (arrival_time_s, Workload)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, size=count)
    t = np.cumsum(gaps) - gaps[0]
    sizes = rng.integers(0, len(SERVE_SIZES), size=count)
    views = rng.integers(0, len(SERVE_VIEWS), size=count)
    out = []
    for i in range(count):
        n, px, nb = SERVE_SIZES[sizes[i]]
        V = SERVE_VIEWS[views[i]]
        out.append((float(t[i]), _wl(f"req{i}_{n}_v{V}", n, px, V, nb, 1000 + i, 8, 4, 2e4,
                                     n_outer=n_outer, n_cg=n_cg)))
    return out


# ---------------------------------------------------------------- phantoms --

@dataclass
class Ellipse:
    cx: float
    cy: float
    a: float      # semi-axis along angle phi
    b: float
    phi: float
    rho: float    # additive attenuation (1/mm)


def random_phantom(geom: Geometry, seed: int, n_ellipses: int, n_disks: int = 0):
    """Seeded ellipse phantom inside the image's inscribed circle.

    Centres are uniform in a disk of radius 0.8*FOV/2, semi-axes 5-40 % of the
    field of view (shrunk so each ellipse stays inside 0.95 of the inscribed
    circle), orientations uniform, densities U(0, 0.02)/mm rescaled so that
    their sum, the worst overlap, is at most 0.02/mm.  Disks have diameters
    2-8 mm and density +0.02/mm.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    fov = geom.n * geom.pixel_mm
    r_in = 0.95 * fov / 2
    out = []
    for _ in range(n_ellipses):
        r = 0.8 * fov / 2 * math.sqrt(rng.random())
        th = 2 * math.pi * rng.random()
        cx, cy = r * math.cos(th), r * math.sin(th)
        a, b = rng.uniform(0.05, 0.40, size=2) * fov
        room = max(r_in - math.hypot(cx, cy), 0.02 * fov)
        s = min(1.0, room / max(a, b))
        out.append(Ellipse(cx, cy, a * s, b * s, math.pi * rng.random(), rng.uniform(0.0, MU_MAX)))
    tot = sum(e.rho for e in out)
    if tot > MU_MAX:
        for e in out:
            e.rho *= MU_MAX / tot
    for _ in range(n_disks):
        r = 0.7 * fov / 2 * math.sqrt(rng.random())
        th = 2 * math.pi * rng.random()
        d = rng.uniform(2.0, 8.0)
        out.append(Ellipse(r * math.cos(th), r * math.sin(th), d / 2, d / 2, 0.0, MU_MAX))
    return out


def ray_lines(geom: Geometry):
    """Source points (V,1,2) and unit directions (V,n_b,2) of every ray."""
    v = np.arange(geom.n_views, dtype=np.float64)
    j = np.arange(geom.n_bins, dtype=np.float64)
    beta = geom.beta0 + geom.arc * v / geom.n_views
    gamma = (j - 0.5 * (geom.n_bins - 1)) * geom.fan_pitch
    src = geom.dso_mm * np.stack([np.cos(beta), np.sin(beta)], axis=-1)[:, None, :]
    theta = beta[:, None] + math.pi + gamma[None, :]
    u = np.stack([np.cos(theta), np.sin(theta)], axis=-1)
    return src, u


def ellipse_line_integrals(geom: Geometry, ellipses) -> np.ndarray:
    """Exact line integrals (V, n_b) of the phantom along every ray.

    Each ray S + t u (|u| = 1) is mapped into the ellipse's frame, the
    quadratic for its two boundary crossings is solved, and the chord length
    (difference of the roots, sqrt(disc)/A) is weighted by the density.
    """
    src, u = ray_lines(geom)
    p = np.zeros((geom.n_views, geom.n_bins))
    for e in ellipses:
        c, s = math.cos(e.phi), math.sin(e.phi)
        # re-origin each ray at its point closest to the ellipse centre, so the
        # quadratic's coefficients stay O(1) instead of O(dso/a)
        rx, ry = src[..., 0] - e.cx, src[..., 1] - e.cy
        tc = rx * u[..., 0] + ry * u[..., 1]
        rx, ry = rx - tc * u[..., 0], ry - tc * u[..., 1]
        qx = rx * c + ry * s
        qy = -rx * s + ry * c
        wx = u[..., 0] * c + u[..., 1] * s
        wy = -u[..., 0] * s + u[..., 1] * c
        A = wx * wx / e.a**2 + wy * wy / e.b**2
        B = 2.0 * (qx * wx / e.a**2 + qy * wy / e.b**2)
        C = qx * qx / e.a**2 + qy * qy / e.b**2 - 1.0
        disc = B * B - 4.0 * A * C
        p += e.rho * np.where(disc > 0, np.sqrt(np.maximum(disc, 0.0)) / A, 0.0)
    return p


@dataclass
class Rect:
    cx: float
    cy: float
    w: float      # side along angle phi
    h: float
    phi: float
    rho: float    # additive attenuation (1/mm)


def rect_line_integrals(geom: Geometry, rects) -> np.ndarray:
    """Exact line integrals (V, n_b) of rectangles: each ray is mapped into a
    rectangle's frame and clipped by its two slabs; the chord times the
    density."""
    src, u = ray_lines(geom)
    p = np.zeros((geom.n_views, geom.n_bins))
    for r in rects:
        c, s = math.cos(r.phi), math.sin(r.phi)
        sx, sy = src[..., 0] - r.cx, src[..., 1] - r.cy
        px, py = sx * c + sy * s, -sx * s + sy * c          # source in the rectangle's frame
        ux, uy = u[..., 0] * c + u[..., 1] * s, -u[..., 0] * s + u[..., 1] * c
        lo = np.full(px.shape, -np.inf)
        hi = np.full(px.shape, np.inf)
        for q, d, half in ((px, ux, 0.5 * r.w), (py, uy, 0.5 * r.h)):
            with np.errstate(divide="ignore", invalid="ignore"):
                t1, t2 = (-half - q) / d, (half - q) / d
            par = d == 0.0
            inside = np.abs(q) < half
            t_lo = np.where(par, np.where(inside, -np.inf, np.inf), np.minimum(t1, t2))
            t_hi = np.where(par, np.where(inside, np.inf, -np.inf), np.maximum(t1, t2))
            lo, hi = np.maximum(lo, t_lo), np.minimum(hi, t_hi)
        p += r.rho * np.maximum(hi - lo, 0.0)
    return p


def shape_line_integrals(geom: Geometry, shapes) -> np.ndarray:
    """Line integrals of a list of Ellipse and Rect shapes."""
    ell = [e for e in shapes if isinstance(e, Ellipse)]
    rec = [r for r in shapes if isinstance(r, Rect)]
    return ellipse_line_integrals(geom, ell) + rect_line_integrals(geom, rec)


# ---------------------------------------------------- evaluation phantoms ----
# Synthetic stand-ins for the paper's image-quality phantom (resolution and
# contrast slices, Figs. 1-4): a water-like disk with bar groups, and one with
# four low-contrast disk targets.
PHANTOM_RADIUS = 150.0   # mm
BAR_LP_CM = (2.0, 3.0, 4.0, 5.0)


def resolution_phantom(n_bars: int = 5, bar_len: float = 20.0, contrast: float = 0.5 * MU_MAX):
    """Disk of MU_MAX with, per frequency in BAR_LP_CM, a group of n_bars bars
    of width 10/(2 lp) mm and period 10/lp mm (vertical bars: the profile runs
    along x), the groups on a ring of 60 mm.  Returns (shapes, groups) with
    groups[lp] = (centre x, centre y, bar width)."""
    shapes = [Ellipse(0.0, 0.0, PHANTOM_RADIUS, PHANTOM_RADIUS, 0.0, MU_MAX)]
    groups = {}
    for k, lp in enumerate(BAR_LP_CM):
        width = 10.0 / (2.0 * lp)
        ang = 2.0 * math.pi * k / len(BAR_LP_CM) + math.pi / 4
        gx, gy = 60.0 * math.cos(ang), 60.0 * math.sin(ang)
        for b in range(n_bars):
            x = gx + (b - (n_bars - 1) / 2) * 2.0 * width
            shapes.append(Rect(x, gy, width, bar_len, 0.0, contrast))
        groups[lp] = (gx, gy, width)
    return shapes, groups


CONTRAST_TARGETS = ((12.0, 0.10), (10.0, 0.05), (8.0, 0.03), (6.0, 0.02))   # (radius mm, relative contrast)


def contrast_phantom():
    """Disk of MU_MAX with four disk targets (ROI 1-4) of decreasing size and
    relative contrast on a ring of 70 mm.  Returns (shapes, rois) with
    rois[i] = (centre x, centre y, radius)."""
    shapes = [Ellipse(0.0, 0.0, PHANTOM_RADIUS, PHANTOM_RADIUS, 0.0, MU_MAX)]
    rois = []
    for k, (r, c) in enumerate(CONTRAST_TARGETS):
        ang = 2.0 * math.pi * k / len(CONTRAST_TARGETS)
        x, y = 70.0 * math.cos(ang), 70.0 * math.sin(ang)
        shapes.append(Ellipse(x, y, r, r, 0.0, c * MU_MAX))
        rois.append((x, y, r))
    return shapes, rois


def noisy_sinogram(p: np.ndarray, photons: float, seed: int) -> np.ndarray:
    """Y = -ln(max(counts, 1)/I0), counts ~ Poisson(I0 exp(-p))."""
    rng = np.random.Generator(np.random.PCG64(seed + 0x5EED))
    counts = rng.poisson(photons * np.exp(-p))
    return -np.log(np.maximum(counts, 1) / photons)


def rasterize(geom: Geometry, ellipses, ss: int = 4) -> np.ndarray:
    """Ground-truth image (n, n) by ss x ss supersampling; reporting only."""
    n, dx = geom.n, geom.pixel_mm
    x0 = -0.5 * n * dx
    off = (np.arange(n * ss) + 0.5) * dx / ss + x0
    X = np.zeros((n * ss, n * ss))
    yy, xx = np.meshgrid(off, off, indexing="ij")
    for e in ellipses:
        c, s = math.cos(e.phi), math.sin(e.phi)
        u = (xx - e.cx) * c + (yy - e.cy) * s
        v = -(xx - e.cx) * s + (yy - e.cy) * c
        if isinstance(e, Rect):
            X += e.rho * ((np.abs(u) <= 0.5 * e.w) & (np.abs(v) <= 0.5 * e.h))
        else:
            X += e.rho * ((u / e.a) ** 2 + (v / e.b) ** 2 <= 1.0)
    return X.reshape(n, ss, n, ss).mean(axis=(1, 3))


def make_case(w: Workload, noise: bool = True):
    """(phantom, noiseless line integrals, measured sinogram Y) of a workload."""
    ell = random_phantom(w.geom, w.seed, w.n_ellipses, w.n_disks)
    p = ellipse_line_integrals(w.geom, ell)
    Y = noisy_sinogram(p, w.photons, w.seed) if noise else p
    return ell, p, Y


def random_image(n: int, seed: int) -> np.ndarray:
    return np.random.Generator(np.random.PCG64(seed)).random((n, n))


def random_sinogram(n_views: int, n_bins: int, seed: int) -> np.ndarray:
    return np.random.Generator(np.random.PCG64(seed)).random((n_views, n_bins))
