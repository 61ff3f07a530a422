"""Pins for the local-AABB count K (App. A uses K = 10 slices per axis;
Tab. 13 ablates 2 and 5): the oracle with K slices against exact clipping,
closed forms at K = 1, the nesting of finer slicings, the conservativeness
of the envelopes and the packing invariants.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from exact_cover import check_packing, cover, placed_polygon
from test_oracle_pins import _assert_cover_inside, _clip_extent, _lshape, local_polygon

R = oracle.R
F = 1 << 18
LAABB_ONLY = oracle.F_ALL & ~oracle.F_OBB


def _charts():
    return (synth.plain64(seed=12, n=14), synth.stars(13, 14, 256, density=1.0))


@pytest.mark.parametrize("K", [1, 2, 3, 5, 7])
def test_slices_match_clipping(K):
    """K equal slices per axis (boundaries floor(i * extent / K)); each
    slice's extent equals an exact Sutherland-Hodgman clip of the
    reoriented chart."""
    params = oracle.default_params(laabb_k=K)
    for cs in _charts():
        rec = oracle.prep(cs, params)
        for i in range(cs.n):
            r = rec[i]
            assert r[R["LK"]] == K
            Wq, Hq = int(r[R["WQ"]]), int(r[R["HQ"]])
            X = r[R["X"]:R["X"] + K + 1]
            Y = r[R["Y"]:R["Y"] + K + 1]
            assert list(X) == [s * Wq // K for s in range(K + 1)]
            assert list(Y) == [s * Hq // K for s in range(K + 1)]
            poly = local_polygon(r, cs.polygon(i))
            for s in range(K):
                assert _clip_extent(poly, int(X[s]), int(X[s + 1]), 0) == (r[R["YLO"] + s], r[R["YHI"] + s])
                assert _clip_extent(poly, int(Y[s]), int(Y[s + 1]), 1) == (r[R["XLO"] + s], r[R["XHI"] + s])


def test_one_slice_is_the_box():
    """K = 1: the one slice per axis is the AABB, so its empty areas are all
    zero (no reflection, App. A) and the local-AABB envelope is the box."""
    params = oracle.default_params(laabb_k=1, flags=LAABB_ONLY)
    for cs in _charts():
        rec = oracle.prep(cs, params)
        assert np.all(rec[:, R["FLIPX"]] == 0) and np.all(rec[:, R["FLIPY"]] == 0)
        for i in range(cs.n):
            for k in (64, 512, 1024):
                e = oracle.envelope(rec[i], k, params)
                assert np.all(e.top == 0) and np.all(e.bot == e.h)
                assert np.all(e.left == 0) and np.all(e.right == e.w)


@pytest.mark.parametrize("coarse", [1, 2, 5])
def test_finer_slicing_nests(coarse):
    """The ten slices refine the two and the five (floor(i E / 2) =
    floor(5 i E / 10), floor(i E / 5) = floor(2 i E / 10)): each fine slice
    lies in a coarse one, so its extent, its refinement by the other axis
    and hence the local-AABB envelope are at least as tight -- wherever the
    chart got the same reflections under both counts."""
    pf = oracle.default_params(laabb_k=10, flags=LAABB_ONLY)
    pc = oracle.default_params(laabb_k=coarse, flags=LAABB_ONLY)
    compared = 0
    for cs in _charts():
        rf, rc = oracle.prep(cs, pf), oracle.prep(cs, pc)
        for i in range(cs.n):
            if (rf[i, R["FLIPX"]], rf[i, R["FLIPY"]]) != (rc[i, R["FLIPX"]], rc[i, R["FLIPY"]]):
                continue
            compared += 1
            for k in (128, 1024):
                ef, ec = oracle.envelope(rf[i], k, pf), oracle.envelope(rc[i], k, pc)
                assert np.all(ef.top >= ec.top) and np.all(ef.bot <= ec.bot)
                assert np.all(ef.left >= ec.left) and np.all(ef.right <= ec.right)
    assert compared >= 5


@pytest.mark.parametrize("K", [2, 5])
@pytest.mark.parametrize("flags", [oracle.F_ALL, LAABB_ONLY])
def test_envelope_contains_exact_cover(K, flags):
    """Conservativeness at every count: the chart's texels lie inside its
    column and row envelopes."""
    params = oracle.default_params(laabb_k=K, flags=flags)
    for cs in _charts():
        rec = oracle.prep(cs, params)
        for i in range(cs.n):
            for k in (64, 400 // 16 * 16, 1024):
                e = oracle.envelope(rec[i], k, params)
                poly, w, h = placed_polygon(cs.polygon(i), k, int(rec[i, R["ROT"]]), int(rec[i, R["FLIPX"]]),
                                            int(rec[i, R["FLIPY"]]), 0)
                cv = cover(poly, w, h)
                assert cv.shape == (e.h, e.w)
                _assert_cover_inside(cv, e)


@pytest.mark.parametrize("K", [2, 5])
@pytest.mark.parametrize("corner", ["tr", "tl", "br", "bl"])
def test_orientation_with_fewer_slices(K, corner):
    """App. A reflections read the empty areas off the slices; two slices
    per axis still see an L's notch and move it to the bottom right."""
    cs = synth.from_polygons([_lshape(corner)], 128, 128)
    rec = oracle.prep(cs, oracle.default_params(laabb_k=K))
    poly = local_polygon(rec[0], cs.polygon(0))
    Wq, Hq = poly[:, 0].max(), poly[:, 1].max()
    assert not any((x == Wq and y == Hq) for x, y in poly)


@pytest.mark.parametrize("K", [2, 5])
def test_pack_invariants(K):
    """Overlap-free, gutters respected, inside the atlas, the largest
    successful candidate returned -- with fewer local AABBs too."""
    cs = synth.knees(4, 150, 512)
    params = oracle.default_params(laabb_k=K)
    r = oracle.pack(cs, params, all_scales=True)
    assert r.status == 0
    rec = oracle.prep(cs, params)
    res = check_packing(cs, r.place[:, 10], r.place, envelope_fn=lambda c, kc: oracle.envelope(rec[c], kc, params))
    assert res == dict(out_of_atlas=0, gutter_overlap=0, overlap=0, outside_envelope=0)
    j = r.k // 16
    assert r.success[j - 1] == 1 and not np.any(r.success[j:])


def test_invalid_count_rejected():
    cs = synth.plain64(seed=1, n=3)
    for K in (0, 11):
        with pytest.raises(ValueError):
            oracle.prep(cs, oracle.default_params(laabb_k=K))


@pytest.mark.parametrize("K", [1, 2, 5])
def test_ten_slot_expansion_is_exact(K):
    """For K dividing 10, slice s of K is the union of ten-slices
    10 s / K .. 10 (s + 1) / K - 1 (floor(s E / K) = floor((10 s / K) E / 10)),
    so a record with ten slots, slot t holding slice t K / 10, gives the same
    envelopes as the K slices (the layout the GPU records use)."""
    params = oracle.default_params(laabb_k=K)
    slot = np.arange(10) * K // 10
    for cs in _charts():
        rec = oracle.prep(cs, params)
        for i in range(cs.n):
            r = rec[i].copy()
            x = r.copy()
            Wq, Hq = int(r[R["WQ"]]), int(r[R["HQ"]])
            x[R["X"]:R["X"] + 11] = [t * Wq // 10 for t in range(11)]
            x[R["Y"]:R["Y"] + 11] = [t * Hq // 10 for t in range(11)]
            for f in ("YLO", "YHI", "XLO", "XHI"):
                x[R[f]:R[f] + 10] = r[R[f] + slot]
            x[R["LK"]] = 10
            for k in (96, 512, 1024):
                a, b = oracle.envelope(r, k, params), oracle.envelope(x, k, params)
                assert np.array_equal(a.top, b.top) and np.array_equal(a.bot, b.bot)
                assert np.array_equal(a.left, b.left) and np.array_equal(a.right, b.right)
