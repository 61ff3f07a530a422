"""Pins for the CPU oracle: each test ties a part of the oracle to something
other than itself -- a constant the paper states, a closed form, a brute-force
search on tiny inputs, or an invariant the paper claims (no overlaps, gutters
respected, every chart inside the atlas, largest successful scale returned).
"""
from __future__ import annotations

import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from exact_cover import F, check_packing, cover, dilate, placed_polygon

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
R = oracle.R
K = oracle.K


def golden():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        return json.load(f)


def local_polygon(rec1, verts):
    """Chart-local Q.8 vertices after rotate/reflect, rebuilt from the flags."""
    q, _, _ = placed_polygon(verts, 1, int(rec1[R["ROT"]]), int(rec1[R["FLIPX"]]),
                             int(rec1[R["FLIPY"]]), 0)
    return q


# ---------------------------------------------------------------------------
# constants the paper states
# ---------------------------------------------------------------------------

def test_paper_constants():
    g = golden()
    p = oracle.default_params()
    assert p[0] == g["gutter_px"]["value"]
    assert p[1] == g["knee_abs_pct_of_atlas_height"]["value"]
    assert p[2] == g["knee_rel_pct_of_taller_chart"]["value"]
    assert p[3] == g["lr_significance_pct_of_aabb_area"]["value"]
    assert oracle.K == g["local_aabbs_per_axis"]["value"]
    C, S = oracle.obb_table()
    assert len(C) == g["obb_angles"]["count"]
    # the 64 candidates k = 16 j are the paper's j/64
    cs = synth.rectangles([(1, 1)], 4, 4)
    r = oracle.pack(cs, all_scales=True)
    assert len(r.success) == g["candidate_scales"]["count"]


def test_obb_table_identities():
    C, S = oracle.obb_table()
    assert (C[0], S[0]) == (16384, 0)
    # cos(m pi/16) = sin((8-m) pi/16)
    for m in range(1, 8):
        assert C[m] == S[8 - m]
    assert C[4] == S[4] == 11585  # 2^14 / sqrt(2) = 11585.24
    # cos(pi/8) = sqrt(2 + sqrt(2)) / 2
    assert C[2] == round(16384 * math.sqrt(2 + math.sqrt(2)) / 2)
    for m in range(8):
        assert abs(int(C[m]) ** 2 + int(S[m]) ** 2 - (1 << 28)) <= 2 * 16384
    # angles increase: S strictly increasing, C strictly decreasing
    assert np.all(np.diff(S) > 0) and np.all(np.diff(C) < 0)


# ---------------------------------------------------------------------------
# prep: AABB, rotation, slices, orientation, OBB
# ---------------------------------------------------------------------------

def test_prep_rectangle_closed_form():
    cs = synth.rectangles([(30, 10), (10, 30), (7, 7)], 64, 64)
    rec = oracle.prep(cs)
    # wider than tall -> rotated to be tall (Sec. 3.1)
    assert rec[0, R["ROT"]] == 1 and rec[0, R["WQ"]] == 10 * 256 and rec[0, R["HQ"]] == 30 * 256
    assert rec[1, R["ROT"]] == 0 and rec[1, R["WQ"]] == 10 * 256 and rec[1, R["HQ"]] == 30 * 256
    assert rec[2, R["ROT"]] == 0  # square: not rotated
    for r in rec:
        Wq, Hq = r[R["WQ"]], r[R["HQ"]]
        X = r[R["X"]:R["X"] + K + 1]
        assert list(X) == [i * Wq // K for i in range(K + 1)]
        assert np.all(r[R["YLO"]:R["YLO"] + K] == 0) and np.all(r[R["YHI"]:R["YHI"] + K] == Hq)
        assert np.all(r[R["XLO"]:R["XLO"] + K] == 0) and np.all(r[R["XHI"]:R["XHI"] + K] == Wq)
        assert r[R["OBBM"]] == 0  # the axis-aligned box is its own minimum box
        assert r[R["U0"]] == 0 and r[R["U1"]] == 16384 * Wq
        assert r[R["FLIPX"]] == 0 and r[R["FLIPY"]] == 0


def _clip_extent(poly, a, b, axis):
    """Independent slab extent: Sutherland-Hodgman clip of the polygon to
    a <= u <= b (u = coordinate `axis`) with exact fractions; floor(min) and
    ceil(max) of the other coordinate over the clipped vertices."""
    pts = [(Fraction(int(p[axis])), Fraction(int(p[1 - axis]))) for p in poly]

    def clip(pts, keep, inter):
        out = []
        for i in range(len(pts)):
            cur, nxt = pts[i], pts[(i + 1) % len(pts)]
            if keep(cur):
                out.append(cur)
                if not keep(nxt):
                    out.append(inter(cur, nxt))
            elif keep(nxt):
                out.append(inter(cur, nxt))
        return out

    def at(u):
        def f(p, q):
            t = (u - p[0]) / (q[0] - p[0])
            return (Fraction(u), p[1] + t * (q[1] - p[1]))
        return f

    pts = clip(pts, lambda p: p[0] >= a, at(Fraction(a)))
    if pts:
        pts = clip(pts, lambda p: p[0] <= b, at(Fraction(b)))
    vs = [p[1] for p in pts]
    return math.floor(min(vs)), math.ceil(max(vs))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_local_aabbs_match_clipping(seed):
    cs = synth.plain64(seed=seed, n=12)
    rec = oracle.prep(cs)
    for i in range(cs.n):
        r = rec[i]
        poly = local_polygon(r, cs.polygon(i))
        X = r[R["X"]:R["X"] + K + 1]
        Y = r[R["Y"]:R["Y"] + K + 1]
        for s in range(K):
            lo, hi = _clip_extent(poly, int(X[s]), int(X[s + 1]), 0)
            assert (lo, hi) == (r[R["YLO"] + s], r[R["YHI"] + s])
            lo, hi = _clip_extent(poly, int(Y[s]), int(Y[s + 1]), 1)
            assert (lo, hi) == (r[R["XLO"] + s], r[R["XHI"] + s])


T = 256  # one texel in Q.8


def _lonly(k=2):
    """Local-AABB proxy alone (no OBB), K slices per axis."""
    return oracle.default_params(laabb_k=k, flags=oracle.F_LAABB | oracle.F_HC | oracle.F_BALANCE)


def test_merge_tightens_columns_closed_form():
    """Sec. 4.1.1: the two sets of local AABBs are merged, each boundary
    taking the tighter bound (the inset uses 2 AABBs per axis).  A staircase
    [0,6]x[0,16] + [6,8]x[10,16] (texels, tall, no reflection) at K = 2:
    x-slice 1 ([4,8]) reaches the top at x in [4,6], so alone it bounds
    every column from 4 to 8 by y = 0; the y-slice [0,8] only spans
    x in [0,6], so columns 6 and 7 meet only the y-slice [8,16] and the
    merged top there is 8 (the true top is 10).  By hand, at scale 1 and
    1/2 (column 3 at 1/2 covers x in (6,8), so floor(8/2) = 4)."""
    poly = [(0, 0), (6 * T, 0), (6 * T, 10 * T), (8 * T, 10 * T), (8 * T, 16 * T), (0, 16 * T)]
    cs = synth.from_polygons([poly], 64, 64)
    p = _lonly()
    rec = oracle.prep(cs, p)
    r = rec[0]
    assert (r[R["ROT"]], r[R["FLIPY"]], r[R["FLIPX"]]) == (0, 0, 0)
    assert list(r[R["YLO"]:R["YLO"] + 2]) == [0, 0]          # the x-slices alone: top 0 everywhere
    assert list(r[R["XHI"]:R["XHI"] + 2]) == [6 * T, 8 * T]
    e = oracle.envelope(r, 1024, p)
    assert list(e.top) == [0, 0, 0, 0, 0, 0, 8, 8]
    assert list(e.bot) == [16] * 8
    assert list(e.right) == [6] * 8 + [8] * 8
    e = oracle.envelope(r, 512, p)
    assert list(e.top) == [0, 0, 0, 4]
    assert list(e.bot) == [8] * 4


def test_merge_tightens_rows_closed_form():
    """The same merge along the other axis: [0,8]x[0,10] + [0,2]x[10,16] at
    K = 2.  The y-slice [8,16] reaches x = 8 (rows 8-9), so alone it bounds
    rows 8-15 by x = 8; the x-slice [4,8] spans only y in [0,10], so rows
    10-15 meet only the x-slice [0,4] and their merged right edge is 4 (the
    true edge is 2).  No reflection: the left and right areas are equal and
    the bottom area lies right of the midline."""
    poly = [(0, 0), (8 * T, 0), (8 * T, 10 * T), (2 * T, 10 * T), (2 * T, 16 * T), (0, 16 * T)]
    cs = synth.from_polygons([poly], 64, 64)
    p = _lonly()
    rec = oracle.prep(cs, p)
    r = rec[0]
    assert (r[R["ROT"]], r[R["FLIPY"]], r[R["FLIPX"]]) == (0, 0, 0)
    assert list(r[R["XHI"]:R["XHI"] + 2]) == [8 * T, 8 * T]  # the y-slices alone: right edge 8
    e = oracle.envelope(r, 1024, p)
    assert list(e.right) == [8] * 10 + [4] * 6
    assert list(e.left) == [0] * 16
    assert list(e.top) == [0] * 8 and list(e.bot) == [16] * 4 + [10] * 4


def test_merge_keeps_every_chart_point_inside():
    """The merged envelope still contains every texel the chart meets, at
    every slice count and with the OBB off (the merge alone decides)."""
    for kk in (2, 5, 10):
        cs = synth.plain64(seed=4, n=16)
        p = _lonly(kk)
        rec = oracle.prep(cs, p)
        for i in range(cs.n):
            for k in (256, 640, 1024):
                r = rec[i]
                e = oracle.envelope(r, k, p)
                poly, w, h = placed_polygon(cs.polygon(i), k, int(r[R["ROT"]]), int(r[R["FLIPX"]]),
                                            int(r[R["FLIPY"]]), 0)
                cv = cover(poly, w, h)
                rr = np.arange(h)[:, None]
                assert not np.any(cv & ~((rr >= e.top[None, :]) & (rr < e.bot[None, :])))
                cc = np.arange(w)[None, :]
                assert not np.any(cv & ~((cc >= e.left[:, None]) & (cc < e.right[:, None])))


def _lshape(notch_corner, W=40, H=60, a=15, b=25):
    """Axis-aligned L: box [0,W]x[0,H] (texels) with a notch of size
    (W-a) x b cut at the given corner ('tr','tl','br','bl'); y grows down."""
    pts = {
        "tr": [(0, 0), (a, 0), (a, b), (W, b), (W, H), (0, H)],
        "tl": [(0, b), (W - a, b), (W - a, 0), (W, 0), (W, H), (0, H)],
        "br": [(0, 0), (W, 0), (W, H - b), (a, H - b), (a, H), (0, H)],
        "bl": [(0, 0), (W, 0), (W, H), (W - a, H), (W - a, H - b), (0, H - b)],
    }[notch_corner]
    return [(x * 256, y * 256) for x, y in pts]


@pytest.mark.parametrize("corner,fy,fx", [("tr", 1, 0), ("tl", 1, 1), ("br", 0, 0), ("bl", 0, 1)])
def test_orientation_moves_empty_area_bottom_right(corner, fy, fx):
    """App. A: reflect vertically if the top empty area exceeds the bottom;
    then horizontally if the left exceeds the right significantly.  An L
    whose notch is at any corner ends with the notch at the bottom right."""
    cs = synth.from_polygons([_lshape(corner)], 128, 128)
    rec = oracle.prep(cs)
    assert rec[0, R["ROT"]] == 0
    assert (rec[0, R["FLIPY"]], rec[0, R["FLIPX"]]) == (fy, fx)
    poly = local_polygon(rec[0], cs.polygon(0))
    # the notch (empty quadrant) now contains the box's bottom-right corner
    xs, ys = poly[:, 0], poly[:, 1]
    Wq, Hq = xs.max(), ys.max()
    assert not any((x == Wq and y == Hq) for x, y in poly)  # corner (Wq,Hq) cut away


def test_orientation_bottom_left_vs_right():
    """App. A tie-break: with equal left/right areas, reflect when the bottom
    area left of the midline exceeds the bottom area right of it."""
    # symmetric-left/right outline: a 'trapezoid' heavier at the bottom-left hole
    W, H = 40, 40
    # triangle whose empty area lies bottom-left: (0,0),(W,0),(W,H)
    cs = synth.from_polygons([[(0, 0), (W * 256, 0), (W * 256, H * 256)]], 128, 128)
    rec = oracle.prep(cs)
    # empty area is bottom-left: bottom > top -> no vertical flip;
    # left > right by > 10 % -> horizontal flip
    assert rec[0, R["FLIPY"]] == 0 and rec[0, R["FLIPX"]] == 1
    # a diamond: left == right and top == bottom -> no flips at all
    cs = synth.from_polygons([[(20 * 256, 0), (40 * 256, 20 * 256), (20 * 256, 40 * 256), (0, 20 * 256)]],
                             128, 128)
    rec = oracle.prep(cs)
    assert rec[0, R["FLIPY"]] == 0 and rec[0, R["FLIPX"]] == 0


def test_obb_finds_table_angle():
    """A rectangle rotated by a table angle is best boxed at that angle, and
    a 45-degree square (exact direction (1,1)) at m = 4."""
    for m in (1, 2, 3, 5, 6):
        th = m * math.pi / 16
        c, s = math.cos(th), math.sin(th)
        w, h = 20 * 256, 60 * 256
        corners = [(0, 0), (w, 0), (w, h), (0, h)]
        # rotate by -theta so that u = xC + yS recovers the rectangle axes
        pts = [(round(x * c - y * s) + 100000, round(x * s + y * c) + 100000) for x, y in corners]
        cs = synth.from_polygons([pts], 512, 512)
        rec = oracle.prep(cs)
        got = int(rec[0, R["OBBM"]])
        # the chart may be reflected, which mirrors the angle: m -> 8 - m (mod 8)
        assert got in (m, (8 - m) % 8), (m, got)
    d = 40 * 256
    cs = synth.from_polygons([[(d, 0), (2 * d, d), (d, 2 * d), (0, d)]], 512, 512)
    assert oracle.prep(cs)[0, R["OBBM"]] == 4


def test_sort_matches_library_stable_sort():
    cs = synth.stars(5, 400, 1024)
    rec = oracle.prep(cs)
    perm = oracle.sort(rec)
    ref = np.lexsort((np.arange(cs.n), -rec[:, R["HQ"]]))
    assert np.array_equal(perm, ref)
    # ties: equal heights keep input order
    cs = synth.rectangles([(3, 5), (4, 5), (2, 9), (1, 5)], 32, 32)
    assert list(oracle.sort(oracle.prep(cs))) == [2, 0, 1, 3]


def test_invalid_inputs_rejected():
    good = synth.rectangles([(3, 5)], 32, 32)
    with pytest.raises(ValueError):
        oracle.prep(synth.from_polygons([[(0, 0), (512, 0)]], 32, 32))  # < 3 vertices
    with pytest.raises(ValueError):
        oracle.prep(synth.from_polygons([[(0, 0), (100, 0), (100, 600)]], 32, 32))  # < 1 texel wide
    with pytest.raises(ValueError):
        oracle.prep(synth.from_polygons([[(0, 0), (1 << 20, 0), (0, 600)]], 32, 32))  # out of range
    assert oracle.pack(good).status == 0
    tiny = synth.rectangles([(300, 300)], 2, 2)  # 300 texels into 2x2: even 1/64 does not fit
    assert oracle.pack(tiny).status == 2


# ---------------------------------------------------------------------------
# envelopes
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("k", [16, 256, 500 // 16 * 16, 1024])
def test_rectangle_envelope_is_the_box(k):
    cs = synth.rectangles([(13, 37), (5, 5)], 64, 64)
    rec = oracle.prep(cs)
    for i in range(2):
        e = oracle.envelope(rec[i], k)
        w = -(-int(rec[i, R["WQ"]]) * k // F)
        h = -(-int(rec[i, R["HQ"]]) * k // F)
        assert (e.w, e.h) == (w, h)
        assert np.all(e.top == 0) and np.all(e.bot == h)
        assert np.all(e.left == 0) and np.all(e.right == w)
        p = oracle.envelope_padded(rec[i], k)
        assert (p.w, p.h) == (w + 2, h + 2)
        assert np.all(p.top == 0) and np.all(p.bot == h + 2)


def _cover_of(cs, rec1, i, k):
    poly, w, h = placed_polygon(cs.polygon(i), k, int(rec1[R["ROT"]]), int(rec1[R["FLIPX"]]),
                                int(rec1[R["FLIPY"]]), 0)
    return cover(poly, w, h)


def _assert_cover_inside(cv, e):
    h, w = cv.shape
    rows = np.arange(h)[:, None]
    cols = np.arange(w)[None, :]
    assert not np.any(cv & ~((rows >= e.top[None, :]) & (rows < e.bot[None, :])))
    assert not np.any(cv & ~((cols >= e.left[:, None]) & (cols < e.right[:, None])))


@pytest.mark.parametrize("flags", [oracle.F_ALL, oracle.F_ALL & ~oracle.F_OBB, oracle.F_ALL & ~oracle.F_LAABB])
def test_envelope_contains_exact_cover(flags):
    """Conservativeness (App. A: the rounding keeps charts separated): every
    texel the chart touches lies inside its column and row envelopes, for
    each proxy alone and for the combination."""
    params = oracle.default_params(flags=flags)
    for cs in (synth.plain64(seed=7, n=20), synth.stars(9, 20, 256, density=1.0)):
        rec = oracle.prep(cs, params)
        for i in range(cs.n):
            for k in (64, 400 // 16 * 16, 1024):
                e = oracle.envelope(rec[i], k, params)
                cv = _cover_of(cs, rec[i], i, k)
                assert cv.shape == (e.h, e.w)
                _assert_cover_inside(cv, e)
                assert np.all((e.top >= 0) & (e.top < e.bot) & (e.bot <= e.h))
                assert np.all((e.left >= 0) & (e.left < e.right) & (e.right <= e.w))


def test_combined_envelope_is_the_tighter_proxy():
    """App. A: per texel, the tighter of the two proxies (larger top,
    smaller bottom)."""
    cs = synth.stars(11, 25, 256, density=1.0)
    pa = oracle.default_params()
    pl = oracle.default_params(flags=oracle.F_ALL & ~oracle.F_OBB)
    po = oracle.default_params(flags=oracle.F_ALL & ~oracle.F_LAABB)
    rec = oracle.prep(cs, pa)
    for i in range(cs.n):
        for k in (128, 1024):
            a, l, o = (oracle.envelope(rec[i], k, p) for p in (pa, pl, po))
            t = np.maximum(l.top, o.top)
            b = np.minimum(l.bot, o.bot)
            ok = b > t  # where the two proxies do not cross, no clamping applies
            assert np.array_equal(a.top[ok], t[ok]) and np.array_equal(a.bot[ok], b[ok])


def test_diamond_envelope_is_exact():
    """A 45-degree square coincides with its m=4 OBB (direction (1,1) is exact
    in the table), so the envelope equals the exact cover's column extents."""
    d = 24 * 256
    cs = synth.from_polygons([[(d, 0), (2 * d, d), (d, 2 * d), (0, d)]], 512, 512)
    rec = oracle.prep(cs)
    for k in (256, 512, 1024):
        e = oracle.envelope(rec[0], k)
        cv = _cover_of(cs, rec[0], 0, k)
        top = cv.argmax(axis=0)
        bot = cv.shape[0] - cv[::-1].argmax(axis=0)
        assert np.array_equal(e.top, top) and np.array_equal(e.bot, bot)
        left = cv.argmax(axis=1)
        right = cv.shape[1] - cv[:, ::-1].argmax(axis=1)
        assert np.array_equal(e.left, left) and np.array_equal(e.right, right)


def test_padded_envelope_contains_dilated_cover():
    cs = synth.plain64(seed=8, n=10)
    rec = oracle.prep(cs)
    for i in range(cs.n):
        for k in (96, 1024):
            p = oracle.envelope_padded(rec[i], k)
            dv = dilate(_cover_of(cs, rec[i], i, k), 1)
            assert dv.shape == (p.h, p.w)
            _assert_cover_inside(dv, p)


# ---------------------------------------------------------------------------
# horizontal compaction and interlock, by brute force
# ---------------------------------------------------------------------------

def _row_bitmap(env, width):
    bm = np.zeros((env.h, width), bool)
    for r in range(env.h):
        bm[r, env.left[r]:env.right[r]] = True
    return bm


def _overlap_at(A, B, dx, dy):
    """Do A's row hulls and B's (shifted right by dx, down by dy) overlap?"""
    W = max(A.w, dx + B.w) + 1
    ba = _row_bitmap(A, W)
    bb = np.zeros_like(ba)
    for r in range(B.h):
        rr = r + dy
        if 0 <= rr < A.h:
            lo, hi = dx + B.left[r], dx + B.right[r]
            bb[rr, max(lo, 0):max(hi, 0)] = True
    return bool(np.any(ba & bb))


@pytest.mark.parametrize("seed", [1, 2])
def test_hcompact_brute_force(seed):
    cs = synth.plain64(seed=seed, n=24)
    rec = oracle.prep(cs)
    perm = oracle.sort(rec)
    for s in range(cs.n - 1):
        a, b = rec[perm[s]], rec[perm[s + 1]]
        for k in (128, 1024):
            A = oracle.envelope_padded(a, k)
            B = oracle.envelope_padded(b, k)
            d, cannot_a, cannot_b = oracle.hcompact(a, b, k)
            # slide B left one texel at a time, top-aligned
            t = 0
            while t + 1 <= A.w and not _overlap_at(A, B, A.w - (t + 1), 0):
                t += 1
            assert d == t
            off = A.w - d
            # B moves up by t relative to A  (B's row r meets A's row r - t)
            b_hit = any(_overlap_at(A, B, off, -u) for u in range(1, B.h + 1))
            # A moves up by t relative to B  (B drops by t relative to A)
            a_hit = any(_overlap_at(A, B, off, u) for u in range(1, A.h + 1))
            assert cannot_b == int(b_hit), (s, k)
            assert cannot_a == int(a_hit), (s, k)


def test_zero_distance_frees_both():
    """App. A: with a compacting distance of zero neither chart is restricted."""
    cs = synth.rectangles([(5, 9), (4, 7)], 64, 64)
    rec = oracle.prep(cs)
    assert oracle.hcompact(rec[0], rec[1], 1024) == (0, 0, 0)


def test_interlock_fixpoint_is_least_solution():
    """Algorithm 2 converges to the least offsets >= the pushed offsets that
    satisfy every restriction; each chart ends at the maximum pushed offset
    over the charts it is chained to."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        n = int(rng.integers(2, 12))
        y0 = rng.integers(0, 50, n)
        ca = rng.integers(0, 2, n).astype(np.uint8)
        cb = rng.integers(0, 2, n).astype(np.uint8)
        ca[-1] = cb[-1] = 0
        y = oracle.correct_y(y0, ca, cb)
        for s in range(n):
            seen, stack = {s}, [s]
            while stack:
                u = stack.pop()
                nxt = []
                if u + 1 < n and ca[u]:
                    nxt.append(u + 1)
                if u - 1 >= 0 and cb[u - 1]:
                    nxt.append(u - 1)
                for v in nxt:
                    if v not in seen:
                        seen.add(v)
                        stack.append(v)
            assert y[s] == max(y0[v] for v in seen)
        for s in range(n - 1):
            if ca[s]:
                assert y[s] >= y[s + 1]
            if cb[s]:
                assert y[s + 1] >= y[s]


# ---------------------------------------------------------------------------
# end to end: closed forms, brute-force reconstruction, invariants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("a,n,W,H", [(10, 30, 64, 64), (7, 50, 100, 60), (16, 9, 50, 50), (3, 200, 128, 40)])
def test_equal_squares_closed_form(a, n, W, H):
    """n equal a x a squares: no knees, no compaction, every direction ties,
    so rows alternate left/right.  With s = ceil(a k / 1024), per_row =
    floor((W+2)/(s+2)), rows = ceil(n / per_row): success iff s <= W and
    rows (s+2) <= H+2, and the placements form the alternating grid."""
    cs = synth.rectangles([(a, a)] * n, W, H)
    r = oracle.pack(cs, all_scales=True)
    exp_k = 0
    for j in range(1, 65):
        k = 16 * j
        s = -(-a * k // 1024)
        ok = s <= W and s <= H
        if ok:
            per = (W + 2) // (s + 2)
            rows = -(-n // per)
            ok = rows * (s + 2) <= H + 2
        assert r.success[j - 1] == int(ok), (k, s)
        if ok:
            exp_k = k
    assert r.k == exp_k
    s = -(-a * exp_k // 1024)
    per = (W + 2) // (s + 2)
    for c in range(n):
        row, col = divmod(c, per)
        x, y, rot, fx, fy, mir = r.place[c, :6]
        assert y == row * (s + 2)
        assert mir == row % 2
        assert x == (col * (s + 2) if row % 2 == 0 else W + 2 - (col + 1) * (s + 2))


def test_single_chart_closed_form():
    cs = synth.stars(21, 1, 256, density=0.3)
    rec = oracle.prep(cs)
    W = H = 37
    cs.atlas_w, cs.atlas_h = W, H
    r = oracle.pack(cs, all_scales=True)
    for j in range(1, 65):
        k = 16 * j
        w = -(-int(rec[0, R["WQ"]]) * k // F)
        h = -(-int(rec[0, R["HQ"]]) * k // F)
        assert r.success[j - 1] == int(w <= W and h <= H)
    assert r.place[0, 0] == 0 and r.place[0, 1] == 0


def _reconstruct_rows(cs, params, r, check_direction=True, knee_check=None):
    """Rebuild, from the placements alone, each row's frontline before the row,
    the drop of every chart onto it (smallest y >= 0 whose padded column
    envelope clears the frontline, found by stepping y), and check each
    chart's final y against the least fixpoint of the drops under the
    interlock restrictions (HC rows) or the drop itself (rows without HC)."""
    rec = oracle.prep(cs, params)
    perm = oracle.sort(rec)
    k = r.k
    d, ca, cb, wp, hp = oracle.scale_pairs(rec, perm, k, params)
    env = [oracle.envelope_padded(rec[perm[s]], k, params) for s in range(cs.n)]
    Wp = cs.atlas_w + 2
    sorted_place = np.zeros((cs.n, 6), np.int64)
    for c in range(cs.n):
        s = r.place[c, 7]
        sorted_place[s] = (r.place[c, 0], r.place[c, 1], r.place[c, 5], r.place[c, 6],
                           r.place[c, 8], r.place[c, 9])
    front = np.zeros(Wp, np.int64)
    prev_dir = 1  # ties on the first row resolve left to right
    nrows = int(sorted_place[:, 3].max()) + 1
    s0 = 0
    for row in range(nrows):
        s1 = s0
        while s1 + 1 < cs.n and sorted_place[s1 + 1, 3] == row:
            s1 += 1
        hc = bool(sorted_place[s0, 4])
        knee = bool(sorted_place[s0, 5])
        mir = int(sorted_place[s0, 2])

        def settle(xs, mirrored):
            drops = []
            for s, X in zip(range(s0, s1 + 1), xs):
                top = env[s].top[::-1] if mirrored else env[s].top
                y = 0
                while np.any(y + top < front[X:X + env[s].w]):  # drop onto the skyline
                    y += 1
                drops.append(y)
            if hc:
                return oracle.correct_y(np.array(drops), ca[s0:s1 + 1].copy(), cb[s0:s1 + 1].copy(),
                                        0, s1 - s0)
            return np.array(drops)

        xs = sorted_place[s0:s1 + 1, 0]
        ys = settle(xs, mir)
        assert np.array_equal(sorted_place[s0:s1 + 1, 1], ys), row
        widths = sum(env[s].w for s in range(s0, s1 + 1))
        if hc and not knee:
            # Sec. 4.2 level 1: compaction is used only if it fits more charts,
            # i.e. the row's charts would not fit side by side
            assert widths > Wp, row
        if knee_check is not None:
            knee_check(row, s0, s1, front, sorted_place, env, Wp)
        if not knee and check_direction:
            # Sec. 4.2 level 2: the other direction, mirrored across the atlas,
            # must not give a smaller maximum frontline (ties alternate)
            alt = np.array([Wp - X - env[s].w for s, X in zip(range(s0, s1 + 1), xs)])
            yalt = settle(alt, 1 - mir)

            def score(xx, yy, mirrored):
                f = front.copy()
                for s, X, y in zip(range(s0, s1 + 1), xx, yy):
                    bot = env[s].bot[::-1] if mirrored else env[s].bot
                    f[X:X + env[s].w] = np.maximum(f[X:X + env[s].w], y + bot)
                return f.max()

            mine, other = score(xs, ys, mir), score(alt, yalt, 1 - mir)
            assert mine <= other, row
            if mine == other:
                assert mir == 1 - prev_dir, row
        prev_dir = mir
        for s in range(s0, s1 + 1):
            X, y, mir = sorted_place[s, :3]
            bot = env[s].bot[::-1] if mir else env[s].bot
            front[X:X + env[s].w] = np.maximum(front[X:X + env[s].w], y + bot)
        s0 = s1 + 1
    assert s0 == cs.n


@pytest.mark.parametrize("make", [lambda: synth.plain64(seed=3), lambda: synth.knees(1, 120, 512),
                                  lambda: synth.stars(4, 150, 512)])
def test_push_reconstructed_from_placements(make):
    cs = make()
    params = oracle.default_params()
    r = oracle.pack(cs, params)
    assert r.status == 0
    _reconstruct_rows(cs, params, r)


WORKLOADS = [
    lambda: synth.plain64(seed=1),
    lambda: synth.plain64(seed=2),
    lambda: synth.stars(3, 300, 512),
    lambda: synth.knees(1, 300, 1024),
    lambda: synth.knees(5, 200, 512),
]


@pytest.mark.parametrize("i", range(len(WORKLOADS)))
def test_invariants_overlap_gutter_bounds(i):
    """Sec. 5 / App. B: outputs are overlap-free, gutters are respected
    (dilated covers disjoint), every chart lies in the atlas; and the
    returned scale succeeds while every larger candidate fails."""
    cs = WORKLOADS[i]()
    r = oracle.pack(cs, all_scales=True)
    assert r.status == 0
    rec = oracle.prep(cs)
    res = check_packing(cs, r.place[:, 10], r.place, envelope_fn=lambda c, kc: oracle.envelope(rec[c], kc))
    assert res == dict(out_of_atlas=0, gutter_overlap=0, overlap=0, outside_envelope=0)
    j = r.k // 16
    assert r.success[j - 1] == 1 and not np.any(r.success[j:])


@pytest.mark.parametrize("flags", [oracle.F_LAABB | oracle.F_OBB,  # balanced off, no HC
                                   oracle.F_ALL & ~oracle.F_BALANCE,
                                   oracle.F_HC | oracle.F_BALANCE,  # boxes only
                                   0])
def test_ablation_modes_keep_invariants(flags):
    cs = synth.knees(2, 150, 512)
    params = oracle.default_params(flags=flags)
    r = oracle.pack(cs, params)
    assert r.status == 0
    rec = oracle.prep(cs, params)
    res = check_packing(cs, r.place[:, 10], r.place, envelope_fn=lambda c, kc: oracle.envelope(rec[c], kc, params))
    assert res == dict(out_of_atlas=0, gutter_overlap=0, overlap=0, outside_envelope=0)


def test_knees_are_detected_and_used():
    """Sec. 4.2: rows following a large height drop fold into the concavity."""
    cs = synth.knees(1, 300, 1024)
    r = oracle.pack(cs)
    assert r.stats[2] >= 1 and r.stats[1] >= 1


def test_tight_and_balanced_help():
    """Tab. 3 direction of effect: the full method reaches a scale at least as
    large as boxes-only with static alternation on these inputs."""
    full, base = [], []
    for seed in range(3):
        cs = synth.knees(seed + 10, 200, 512)
        full.append(oracle.pack(cs).k)
        base.append(oracle.pack(cs, oracle.default_params(flags=0)).k)
    assert sum(full) > sum(base)


def _diamond(W, H):
    W, H = W * 256, H * 256
    return [(W // 2, 0), (W, H // 2), (W // 2, H), (0, H // 2)]


def _rows_sorted(place):
    """(X, mirror, row, w') per sorted position from oracle.pack_scale output."""
    return place


def test_compaction_never_reaches_past_a_neighbour():
    """READING added to Algorithm 4: with compacting on, chart s+2 never
    starts left of chart s's right edge, so only neighbours share columns and
    the pairwise interlock of Algorithm 2 suffices.  Two small diamonds nest
    into a tall diamond's empty upper-right triangle; in a 78-texel atlas
    compaction is what lets the third chart into the row, and the third
    chart's compacted position (57) is clamped to the first chart's right
    edge (62)."""
    cs = synth.from_polygons([_diamond(60, 100), _diamond(10, 20), _diamond(10, 10)], 78, 300)
    rec = oracle.prep(cs)
    perm = oracle.sort(rec)
    d, ca, cb, wp, hp = oracle.scale_pairs(rec, perm, 1024)
    ok, pl, st = oracle.pack_scale(rec, perm, 78, 300, 1024)
    assert ok and list(pl[:, 3]) == [0, 0, 0]
    x = pl[:, 0]
    assert x[1] == wp[0] - d[0] < wp[0]           # compacted into the first box
    assert x[1] + wp[1] - d[1] < x[0] + wp[0]     # plain compaction would reach further
    assert x[2] == x[0] + wp[0]                   # ... and is clamped


@pytest.mark.parametrize("i", range(len(WORKLOADS)))
def test_only_neighbours_share_columns(i):
    cs = WORKLOADS[i]()
    rec = oracle.prep(cs)
    perm = oracle.sort(rec)
    r = oracle.pack(cs)
    d, ca, cb, wp, hp = oracle.scale_pairs(rec, perm, r.k)
    ok, pl, st = oracle.pack_scale(rec, perm, cs.atlas_w, cs.atlas_h, r.k)
    assert ok
    for s in range(cs.n - 2):
        if pl[s, 3] == pl[s + 2, 3]:
            lo0, hi0 = pl[s, 0], pl[s, 0] + wp[s]
            lo2, hi2 = pl[s + 2, 0], pl[s + 2, 0] + wp[s + 2]
            assert hi0 <= lo2 or hi2 <= lo0


@pytest.mark.parametrize("a,b,knee", [(50, 40, 1), (50, 41, 0), (60, 50, 0), (60, 48, 1), (55, 44, 1),
                                      (40, 31, 0), (40, 30, 1), (30, 21, 0)])
def test_knee_thresholds_exact(a, b, knee):
    """App. A: a consecutive height drop is a knee iff it is at least 10 % of
    the atlas height AND at least 20 % of the taller chart (unscaled heights).
    Atlas 100 x 100, one 20 x a rectangle then three 20 x b: one row."""
    cs = synth.rectangles([(20, a)] + [(20, b)] * 3, 100, 100)
    rec = oracle.prep(cs)
    perm = oracle.sort(rec)
    ok, pl, st = oracle.pack_scale(rec, perm, 100, 100, 1024)
    assert ok and st[0] == 1
    assert st[2] == knee


def test_knee_region_follows_the_frontline():
    """Algorithm 3: while rows fold into a knee, the concavity edge moves to
    just past the last texel of the knee chart whose frontline reaches the
    height at the current edge (restated as a sequential scan), and each
    knee-folded row starts at the concavity's near edge.  The knee chart is
    the taller chart of the largest qualifying drop (App. A thresholds) in
    the last full-width row."""
    checked = []
    for seed in range(1, 6):
        cs = synth.knees(seed, 300, 1024)
        params = oracle.default_params()
        r = oracle.pack(cs, params)
        rec = oracle.prep(cs, params)
        perm = oracle.sort(rec)
        hq = rec[perm, R["HQ"]]
        state = {}

        def knee_check(row, s0, s1, front, sp, env, Wp):
            knee = bool(sp[s0, 5])
            if knee:
                kd = state["knee"]
                assert kd is not None
                ltr, L, Rr = kd
                if ltr:  # concavity to the right of the knee chart
                    cur = front[Rr]
                    x = Rr
                    while x - 1 >= L and front[x - 1] < cur:
                        x -= 1
                    Rr = x
                    lo, hi = Rr, Wp
                else:
                    cur = front[L - 1]
                    x = L
                    while x < Rr and front[x] < cur:
                        x += 1
                    L = x
                    lo, hi = 0, L
                state["knee"] = (ltr, L, Rr)
                xs = sp[s0:s1 + 1, 0]
                ws = np.array([env[s].w for s in range(s0, s1 + 1)])
                assert xs.min() >= lo and (xs + ws).max() <= hi, row
                if sp[s0, 2] == 0:
                    assert xs[0] == lo, row
                else:
                    assert xs[0] + ws[0] == hi, row
                checked.append(seed)
            else:
                best, bestD = -1, 0
                for s in range(s0, s1):
                    D = int(hq[s - 0] - hq[s + 1])
                    if 10 * D >= 256 * cs.atlas_h and 5 * D >= int(hq[s]) and D > bestD:
                        best, bestD = s, D
                state["knee"] = None
                if best >= 0:
                    X, w = int(sp[best, 0]), env[best].w
                    ltr = sp[s0, 2] == 0
                    if (ltr and X + w < Wp) or (not ltr and X > 0):
                        state["knee"] = (ltr, X, X + w)

        _reconstruct_rows(cs, params, r, knee_check=knee_check)
    assert len(checked) >= 3
