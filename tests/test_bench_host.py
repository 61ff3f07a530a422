"""Host-side pieces of the benchmark's measurement: the waves a batch runs
for one atlas (the launch count and the algorithmic bytes follow from
them), the algorithmic bytes themselves on a closed-form case, and the
per-word operation count of the raster roofline."""
from __future__ import annotations

import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


@pytest.mark.parametrize("jtop,k_best,F", [(40, 512, 2), (63, 1024, 8), (10, 16, 3), (5, 0, 2), (30, 496, 64)])
def test_wave_ranges(jtop, k_best, F):
    waves = bench.wave_ranges(jtop, k_best, F)
    j_best = k_best // 16 - 1 if k_best else -1
    seen = [j for _, js in waves for j in js]
    # each wave below the one before it, together every candidate from the
    # top one down, F per wave but the last
    assert all(waves[w][1][0] > waves[w + 1][1][-1] for w in range(len(waves) - 1))
    assert max(seen) == jtop and sorted(seen) == list(range(min(seen), jtop + 1))
    assert all(len(js) == F for _, js in waves[:-1])
    assert [w for w, _ in waves] == list(range(len(waves)))
    if j_best >= 0:
        assert j_best in waves[-1][1]  # the search stops in the wave of its result
    else:
        assert min(seen) == 0  # no success: every candidate down to the smallest


def test_algorithmic_bytes_closed_form():
    """Equal squares of side a texels: at candidate k each has w' = h' =
    ceil(a k / 1024) + 2g, so the raster writes 4 (w' + h') B per chart (4 B
    per padded scanline word) and the compactor reads 4 h' B plus 25 B per
    chart."""
    a, n = 7, 5
    cs = synth.rectangles([(a, a)] * n, 64, 64)
    jtop, k_best, F = 63, 1024, 1
    got = bench.algorithmic_bytes([cs], [k_best], [jtop], F)
    wp = -(-a * 1024 // 1024) + 2
    assert got["raster"] == n * 8 * wp
    assert got["hcompact"] == n * (4 * wp + 25)


def test_raster_ops_per_word():
    assert bench.raster_ops_per_word(1) == 120
    assert bench.raster_ops_per_word(0) == 116 and bench.raster_ops_per_word(2) == 124


def test_p99_crossing_rate():
    """Linear in p99 over log(rate) between the bracketing rates."""
    c = bench.crossing([(1000, 5.0), (2000, 10.0), (4000, 20.0), (8000, 40.0)])
    assert c["between"] == [2000, 4000]
    assert abs(c["rate"] - 2000 * 2 ** 0.5) < 0.1
    assert bench.crossing([(1000, 16.0), (2000, 30.0)])["rate"] is None
    assert bench.crossing([(1000, 1.0), (2000, 3.0)])["rate"] is None
