"""Image-quality comparison of FBP, IR and AIR (Results, Tables 1-2) on synthetic
phantoms.

The paper scores reconstructions of an image-quality phantom scanned on a
TomoTherapy MVCT by the FWHM of the 3 lp/cm bars (Table 1) and the CNR of four
low-contrast ROIs (Table 2), each from 100 % (800) and 25 % (200) of the views.
The scans are not available; this module runs the same comparison on the
synthetic bar-group and contrast phantoms of `inputs` with the paper's imaging
geometry (350 x 350 pixels of 1 mm, 528 bins).  The numbers are the synthetic
stand-ins', not the paper's.

Definitions (the paper names the quantities, not their estimators):
* FWHM of a bar group: on the profile across the bars (the image averaged over
  the middle of the bars' length, sampled along x), each inner bar's width at
  half height between its peak and the mean of its two neighbouring valleys,
  by linear interpolation between samples; the mean over the inner bars.
* CNR = |mu_t - mu_b| / sqrt(sigma_t^2 + sigma_b^2) (Results), with the
  target the pixels within 0.7 r of a target disk of radius r and the
  background the annulus 1.5 r .. 2.5 r around it.
* IR = the same split-Bregman solve without the filter (C = I), with mu
  scaled by ||A^T A|| / ||A'^T A|| (power iterations) so that the L2 step
  weighs the data and the split term alike for both.  Each method's lambda is
  the one of LAMBDA_GRID (relative to mu) that gives the lowest RMSE against
  the known contrast phantom, chosen per method and per view count; the
  tables then score those reconstructions.

    python -m paper_1310_1434_gb300.evaluate [--n 350] [--iters 30x8]
"""
from __future__ import annotations

import argparse
import dataclasses
import math

import numpy as np

from . import inputs

# The paper's imaging geometry (Materials): 350 x 350 pixels of 1 mm, 528 bins.
EVAL_GEOM = inputs.Geometry(350, 1.0, 800, 528)
VIEWS = {"100% data": 800, "25% data": 200}
LAMBDA_GRID = (1e-4, 3e-4, 1e-3, 3e-3, 1e-2)   # lambda / mu


# ---------------------------------------------------------------- metrics ----
def half_max_width(profile: np.ndarray, dx: float, centre: int, baseline: float) -> float:
    """Width of the peak at index `centre` at half height between its value
    and `baseline`, the crossings found by linear interpolation."""
    p = np.asarray(profile, dtype=np.float64)
    half = 0.5 * (p[centre] + baseline)
    i = centre
    while i > 0 and p[i - 1] > half:
        i -= 1
    if i == 0:
        return float("nan")
    left = (i - 1) + (half - p[i - 1]) / (p[i] - p[i - 1])
    k = centre
    while k < len(p) - 1 and p[k + 1] > half:
        k += 1
    if k == len(p) - 1:
        return float("nan")
    right = k + (p[k] - half) / (p[k] - p[k + 1])
    return float((right - left) * dx)


def bar_fwhm(profile: np.ndarray, dx: float, x0: float, centres, width: float, inner=None) -> float:
    """Mean FWHM of the bars at positions `centres` (mm) of bar width `width`
    on a profile sampled at x0 + i dx: each bar's peak (the maximum within
    half a bar width of its centre) against the mean of the minima of the two
    gaps beside it."""
    p = np.asarray(profile, dtype=np.float64)
    idx = lambda x: int(round((x - x0) / dx))
    half_w = max(1, int(round(0.5 * width / dx)))
    out = []
    sel = range(1, len(centres) - 1) if inner is None else inner
    for b in sel:
        c = idx(centres[b])
        lo, hi = max(c - half_w, 0), min(c + half_w + 1, len(p))
        peak = lo + int(np.argmax(p[lo:hi]))
        gl, gr = idx(centres[b] - width), idx(centres[b] + width)
        vl = p[max(gl - half_w, 0):gl + half_w + 1].min()
        vr = p[gr - half_w:min(gr + half_w + 1, len(p))].min()
        out.append(half_max_width(p, dx, peak, 0.5 * (vl + vr)))
    return float(np.mean(out))


def cnr(image: np.ndarray, target: np.ndarray, background: np.ndarray) -> float:
    """|mu_t - mu_b| / sqrt(sigma_t^2 + sigma_b^2) over the two masks."""
    t, b = image[target], image[background]
    return float(abs(t.mean() - b.mean()) / math.sqrt(t.var() + b.var()))


def pixel_centres(g: inputs.Geometry):
    c = (np.arange(g.n) + 0.5 - 0.5 * g.n) * g.pixel_mm
    return np.meshgrid(c, c)          # X[iy, ix], Y[iy, ix]


def roi_masks(g: inputs.Geometry, x: float, y: float, r: float):
    X, Y = pixel_centres(g)
    d = np.hypot(X - x, Y - y)
    return d < 0.7 * r, (d > 1.5 * r) & (d < 2.5 * r)


def bar_profile(g: inputs.Geometry, image: np.ndarray, gx: float, gy: float, n_bars: int, width: float,
                bar_len: float):
    """Profile across a bar group (averaged over the middle half of the bars'
    length) and the bars' centre positions, on the pixel grid along x."""
    X, Y = pixel_centres(g)
    rows = np.abs(Y[:, 0] - gy) < 0.25 * bar_len
    span = (n_bars + 1) * 2.0 * width
    cols = np.abs(X[0] - gx) < 0.5 * span
    prof = image[rows][:, cols].mean(axis=0)
    x0 = X[0][cols][0]
    centres = [gx + (b - (n_bars - 1) / 2) * 2.0 * width for b in range(n_bars)]
    return prof, x0, centres


# ------------------------------------------------------------ comparison ----
def operator_norm(air, plan, filtered: bool, iters: int = 12) -> float:
    """||A^T A|| (filtered = False) or ||A'^T A|| (power iteration on the GPU)."""
    import torch
    g = plan.geom
    x = torch.randn(g.n * g.n, device="cuda")
    x /= x.norm()
    y = torch.empty(g.n_views * g.n_bins, device="cuda")
    z = torch.empty_like(x)
    lam = 1.0
    for _ in range(iters):
        air.air_project(plan, x, y)
        (air.air_filtered_backproject if filtered else air.air_backproject)(plan, y, z)
        lam = float(z.norm())
        x = z / lam
    return lam


def solve(air, g: inputs.Geometry, Yd, lam: float, mu: float, n_outer: int, n_cg: int) -> np.ndarray:
    import torch
    X = torch.empty(g.n * g.n, device="cuda")
    air.air_solve(air.Plan(g), Yd, lam, mu, n_outer, n_cg, X)
    return X.cpu().numpy().reshape(g.n, g.n).astype(np.float64)


def evaluate(n: int = 350, pixel_mm: float = 1.0, n_bins: int = 528, views=None, photons: float = 2e4,
             mu: float = 1.0, n_outer: int = 30, n_cg: int = 8, seed: int = 21, grid=LAMBDA_GRID):
    """Tables 1 and 2 on the synthetic phantoms: {"fwhm": {data: {method:
    mm}}, "cnr": {data: {method: [ROI1..4]}}, "lambda": {data: {method: lambda/mu}}}."""
    import torch
    from . import air
    air.load()
    views = VIEWS if views is None else views
    bars, groups = inputs.resolution_phantom()
    targets, rois = inputs.contrast_phantom()
    table1, table2, chosen = {}, {}, {}
    dev = lambda Y: torch.as_tensor(np.ascontiguousarray(Y, dtype=np.float32).ravel(), device="cuda")
    for label, V in views.items():
        g = inputs.Geometry(n, pixel_mm, V, n_bins)
        gi = dataclasses.replace(g, filter=0)
        s = operator_norm(air, air.Plan(gi), False) / operator_norm(air, air.Plan(g), True)
        Yb = dev(inputs.noisy_sinogram(inputs.shape_line_integrals(g, bars), photons, seed))
        Yc = dev(inputs.noisy_sinogram(inputs.shape_line_integrals(g, targets), photons, seed + 1))
        truth = inputs.rasterize(g, targets)
        rb, rc = {}, {}
        X = torch.empty(n * n, device="cuda")
        air.air_fbp(air.Plan(g), Yb, X)
        rb["FBP"] = X.cpu().numpy().reshape(n, n).astype(np.float64)
        air.air_fbp(air.Plan(g), Yc, X)
        rc["FBP"] = X.cpu().numpy().reshape(n, n).astype(np.float64)
        chosen[label] = {}
        for m, gm, scale in (("IR", gi, s), ("AIR", g, 1.0)):
            best = None
            for t in grid:                       # lambda / mu by RMSE on the contrast phantom
                img = solve(air, gm, Yc, t * mu * scale, mu * scale, n_outer, n_cg)
                err = float(np.sqrt(np.mean((img - truth) ** 2)))
                if best is None or err < best[0]:
                    best = (err, t, img)
            chosen[label][m] = best[1]
            rc[m] = best[2]
            rb[m] = solve(air, gm, Yb, best[1] * mu * scale, mu * scale, n_outer, n_cg)
        gx, gy, w = groups[3.0]
        table1[label], table2[label] = {}, {}
        for m in ("FBP", "IR", "AIR"):
            prof, x0, centres = bar_profile(g, rb[m], gx, gy, 5, w, 20.0)
            table1[label][m] = bar_fwhm(prof, pixel_mm, x0, centres, w)
            table2[label][m] = [cnr(rc[m], *roi_masks(g, x, y, r)) for (x, y, r) in rois]
    return {"fwhm": table1, "cnr": table2, "lambda_over_mu": chosen,
            "setup": {"n": n, "pixel_mm": pixel_mm, "n_bins": n_bins, "photons": photons, "mu": mu,
                      "iterations": f"{n_outer}x{n_cg}", "ir_mu_scale": "||A^T A|| / ||A'^T A||"}}


def format_tables(res) -> str:
    lines = ["Table 1 (synthetic): FWHM (mm) of the 3 lp/cm bars", "", "|  | FBP | IR | AIR |", "|---|---|---|---|"]
    for label, row in res["fwhm"].items():
        lines.append(f"| {label} | " + " | ".join(f"{row[m]:.2f}" for m in ("FBP", "IR", "AIR")) + " |")
    if "lambda_over_mu" in res:
        lines += ["", "lambda / mu chosen by RMSE: " + "; ".join(
            f"{label}: IR {v['IR']:g}, AIR {v['AIR']:g}" for label, v in res["lambda_over_mu"].items())]
    lines += ["", "Table 2 (synthetic): CNR of ROI 1-4", "", "|  |  | ROI1 | ROI2 | ROI3 | ROI4 |",
              "|---|---|---|---|---|---|"]
    for label, rows in res["cnr"].items():
        for k, m in enumerate(("FBP", "IR", "AIR")):
            lines.append(f"| {label if k == 0 else ''} | {m} | " + " | ".join(f"{v:.2f}" for v in rows[m]) + " |")
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n", type=int, default=350)
    ap.add_argument("--iters", default="30x8", help="outer x CG iterations")
    args = ap.parse_args()
    n_outer, n_cg = (int(v) for v in args.iters.split("x"))
    print(format_tables(evaluate(n=args.n, n_outer=n_outer, n_cg=n_cg)))


if __name__ == "__main__":
    main()
