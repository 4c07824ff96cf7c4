"""The synthetic image-quality comparison (Tables 1-2 stand-in): its phantom
line integrals and its metrics against closed forms (CPU), and one run of the
comparison on the GPU (pytest -m gpu)."""
import math

import numpy as np
import pytest

from dense import chord
from paper_1310_1434_gb300 import evaluate as ev
from paper_1310_1434_gb300 import inputs


def test_rect_line_integrals_are_slab_chords():
    g = inputs.Geometry(64, 2.0, 12, 41)
    rects = [inputs.Rect(10.0, -5.0, 30.0, 8.0, 0.0, 0.01), inputs.Rect(-20.0, 15.0, 12.0, 40.0, 0.6, 0.02)]
    p = inputs.rect_line_integrals(g, rects)
    src, u = inputs.ray_lines(g)
    for v in range(g.n_views):
        for j in range(0, g.n_bins, 3):
            S, d = src[v, 0], u[v, j]
            ref = 0.0
            for r in rects:   # chord in the rectangle's frame, as an axis-aligned box
                c, s = math.cos(r.phi), math.sin(r.phi)
                Sr = ((S[0] - r.cx) * c + (S[1] - r.cy) * s, -(S[0] - r.cx) * s + (S[1] - r.cy) * c)
                dr = (d[0] * c + d[1] * s, -d[0] * s + d[1] * c)
                ref += r.rho * chord(Sr, dr, -r.w / 2, r.w / 2, -r.h / 2, r.h / 2)
            assert p[v, j] == pytest.approx(ref, abs=1e-12)


def test_bar_phantom_frequencies():
    shapes, groups = inputs.resolution_phantom()
    for lp, (gx, gy, w) in groups.items():
        assert w == pytest.approx(10.0 / (2 * lp))
        bars = sorted(r.cx for r in shapes if isinstance(r, inputs.Rect) and abs(r.cy - gy) < 1e-9 and
                      abs(r.w - w) < 1e-12)
        assert len(bars) == 5
        assert np.allclose(np.diff(bars), 10.0 / lp)          # period of lp line pairs per cm


def test_half_max_width_of_a_gaussian():
    dx, sigma = 0.01, 0.7
    x = np.arange(-800, 801) * dx
    prof = 3.0 * np.exp(-x ** 2 / (2 * sigma ** 2)) + 0.5
    assert ev.half_max_width(prof, dx, 800, 0.5) == pytest.approx(2 * math.sqrt(2 * math.log(2)) * sigma, rel=1e-4)


def test_bar_fwhm_of_sharp_bars_is_the_bar_width():
    dx, w = 0.01, 1.6
    centres = [(b - 2) * 2 * w for b in range(5)]
    x = np.arange(-2000, 2001) * dx
    prof = sum(((np.abs(x - c) < w / 2).astype(float)) for c in centres)
    assert ev.bar_fwhm(prof, dx, x[0], centres, w) == pytest.approx(w, abs=2 * dx)


def test_cnr_of_known_statistics():
    img = np.zeros((4, 100))
    tgt = np.zeros_like(img, bool)
    bkg = np.zeros_like(img, bool)
    tgt[0:2] = True
    bkg[2:4] = True
    img[0] = 1.1
    img[1] = 0.9            # target: mean 1, std 0.1
    img[2] = 0.2
    img[3] = -0.2           # background: mean 0, std 0.2
    assert ev.cnr(img, tgt, bkg) == pytest.approx(1.0 / math.sqrt(0.01 + 0.04), rel=1e-12)


@pytest.mark.gpu
def test_comparison_runs_on_the_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    res = ev.evaluate(n_outer=2, n_cg=2, grid=(1e-3,))   # few iterations: IR and AIR are far from converged
    for label in ev.VIEWS:
        # FBP is a complete reconstruction: the 1.67 mm bars come out near
        # their width on 1 mm pixels
        assert 1.2 < res["fwhm"][label]["FBP"] < 3.0
        for m in ("FBP", "IR", "AIR"):
            assert isinstance(res["fwhm"][label][m], float)
            assert len(res["cnr"][label][m]) == 4 and all(np.isfinite(res["cnr"][label][m]))
    assert "Table 1" in ev.format_tables(res)
