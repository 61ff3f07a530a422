"""The oracle's candidates spread over host cores give the sequential
oracle's result (the multi-core CPU baseline runs this driver), and the
per-chart loop areas weigh the area-weighted choice of Sec. 4.4."""
import numpy as np
import pytest

import oracle
import synth
from oracle import parallel


@pytest.fixture(scope="module")
def ex():
    oracle.build()
    with parallel.pool(2) as e:
        yield e


def test_chart_area2_closed_form():
    sizes = [(3, 5), (7, 2), (1, 1), (40, 9)]
    cs = synth.rectangles(sizes, 64, 64)
    a = oracle.chart_area2(cs)
    assert a.tolist() == [2 * w * h * 256 * 256 for w, h in sizes]


def test_score_is_area_times_scale():
    cs = synth.stars(3, 300, 512)
    r = oracle.pack(cs)
    a = oracle.chart_area2(cs).astype(object)
    assert int((a * r.place[:, 10].astype(object)).sum()) == r.score


@pytest.mark.parametrize("width", [1, 3, 8])
def test_parallel_equals_sequential(ex, width):
    for cs in (synth.plain64(), synth.stars(11, 400, 512)):
        r = oracle.pack(cs)
        st, k, place, perm = parallel.pack_parallel(cs, ex, width)
        assert st == r.status and k == r.k
        assert np.array_equal(place[:, 0], r.place[perm, 0])
        assert np.array_equal(place[:, 1], r.place[perm, 1])
