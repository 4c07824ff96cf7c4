"""Host-side pieces of bench.py that feed the reported numbers (CPU only)."""
import os
import sys

import numpy as np

import oracle
from paper_1310_1434_gb300 import inputs

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_segment_count_matches_the_oracle_siddon_walk():
    """The roofline's work figure nnz(A) equals the number of positive-length
    segments the oracle's Siddon walk produces, summed over rays, up to the
    rays that pass through a grid vertex (the count adds one cell there; the
    central rays of this odd-bin geometry cross the image centre)."""
    w = inputs._wl("seg", 24, 1.3, 30, 41, 3, 4, 2, 1e5)
    g = w.geom
    nnz = 0
    for v in range(g.n_views):
        for j in range(g.n_bins):
            _, ln = oracle.ray_segments(g, v, j)
            nnz += int(np.count_nonzero(ln > 1e-12))
    assert abs(bench.segment_count(g) - nnz) <= 1e-3 * nnz


def test_segment_count_scales_with_views():
    g8 = inputs.AIR512_V800.geom
    g2 = inputs.AIR512_V200.geom
    a, b = bench.segment_count(g8), bench.segment_count(g2)
    assert abs(a / b - 4.0) < 0.01
    # every ray of this geometry crosses the image: at least n pixels each on average
    assert a > g8.n_views * g8.n_bins * 0.5 * g8.n
