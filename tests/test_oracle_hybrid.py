"""Pins for the oracle's prefix-sum tail (Sec. 4.4 "Performance
Optimization", Tab. 4): where the switch happens, a skyline brute force on
boxes (whose envelopes are the boxes themselves and whose compacting
distances are zero), the tightness of the compacted prefix fold, FastAtlas's
direction pattern, and the packing invariants with the tail on.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from exact_cover import check_packing

R = oracle.R


def _ceil_div(a, b):
    return -(-a // b)


def _rows_modulo(P, Wp):
    """Tail rows of the prefix fold: maximal runs of charts with the same
    floor(P / W')."""
    rows = []
    for s, p in enumerate(P):
        if not rows or p // Wp != P[rows[-1][-1]] // Wp:
            rows.append([])
        rows[-1].append(s)
    return rows


def skyline_tail(sizes, W, H, S, g=1):
    """Independent brute force for boxes folded entirely by the tail
    (Sec. 4.4): sorted by height, padded widths at the candidate S, the
    prefix of the widths (boxes have compacting distance 0) cut into rows
    modulo W'; the intermediate scale is the largest k' in S - 14 .. S at
    which every row's widths sum to at most W' (if there is none the tail is
    not taken: (None, 0, {})); rows in FastAtlas's directions (left, right,
    right, ...) from their near end, each box dropped onto the skyline.
    Returns (success, k', {sorted pos: (X, y, mirror, tail row)}).  Boxes
    wider than tall are turned upright first (Sec. 3.1)."""
    sizes = [(min(w, h), max(w, h)) for w, h in sizes]
    order = sorted(range(len(sizes)), key=lambda i: -sizes[i][1])  # stable
    Wp, Hp = W + 2 * g, H + 2 * g

    def wp(k):
        return [_ceil_div(sizes[i][0] * k, 1024) + 2 * g for i in order]

    def hp(k):
        return [_ceil_div(sizes[i][1] * k, 1024) + 2 * g for i in order]

    w = wp(S)
    P = np.concatenate([[0], np.cumsum(w)[:-1]]).astype(int)
    rows = _rows_modulo(P, Wp)
    kt = 0
    for k2 in range(S, max(0, S - 15), -1):
        if all(sum(wp(k2)[s] for s in row) <= Wp for row in rows):
            kt = k2
            break
    if not kt:
        return None, 0, {}
    w2, h2 = wp(kt), hp(kt)
    front = np.zeros(Wp, np.int64)
    out = {}
    for t, row in enumerate(rows):
        mirror = t % 3 != 0
        x, drops = 0, []
        for s in row:
            X = Wp - x - w2[s] if mirror else x
            drops.append((s, X, int(front[X:X + w2[s]].max())))
            x += w2[s]
        for s, X, y in drops:
            front[X:X + w2[s]] = np.maximum(front[X:X + w2[s]], y + h2[s])
            out[s] = (X, y, int(mirror), t)
        if front.max() > Hp:
            return False, kt, out
    return True, kt, out


def _area2(sizes):
    return [2 * (w * 256) * (h * 256) for w, h in sizes]


def _wide_boxes(seed):
    rng = np.random.default_rng(seed)
    return [(int(w), int(w + rng.integers(5, 60))) for w in rng.integers(80, 121, 24)]


# (sizes in texels, atlas W, H): small boxes (whose overflowing rows no
# downscale within a grid step can fix: the rows go on one by one) and boxes
# wide enough that one step of downscale narrows each by a texel
BOXES = [([(3, 5), (2, 2), (4, 6), (1, 3), (5, 5), (2, 4), (3, 3), (1, 1), (2, 6), (4, 4)] * 3, 17, 40),
         ([(1, 2), (2, 3), (3, 3), (1, 1)] * 9 + [(6, 7), (5, 8)], 17, 40),
         ([(9, 11), (7, 9), (8, 8), (6, 10), (5, 7), (9, 6), (4, 9), (8, 5)] * 4, 41, 40),
         (_wide_boxes(7), 520, 900),
         (_wide_boxes(8), 520, 900)]


@pytest.mark.parametrize("case", range(len(BOXES)))
@pytest.mark.parametrize("k", [256, 512, 768, 1024])
@pytest.mark.parametrize("g", [1, 0, 2])
def test_boxes_match_skyline_brute_force(case, k, g):
    sizes, W, H = BOXES[case]
    cs = synth.rectangles(sizes, W, H)
    params = oracle.default_params(topt=1000, hybrid_min=0, gutter=g)  # every row is a tail row
    rec = oracle.prep(cs, params)
    perm = oracle.sort(rec)
    ok, place, stats = oracle.pack_scale(rec, perm, W, H, k, params)
    bok, kt, exp = skyline_tail(sizes, W, H, k, g)
    if bok is None:  # no tail scale within one grid step: the rows are folded one by one
        assert stats[6] == 0 and stats[5] == 0 and stats[7] == cs.n
        assert not np.any(place[:int(stats[4]), 5] == 2)
        return
    assert ok == bok
    assert stats[6] == kt and stats[7] == 0
    placed = int(stats[4])
    assert stats[5] == stats[0]  # all rows are tail rows
    assert placed == len(exp)
    for s in range(placed):
        X, y, mirror, t = exp[s]
        assert tuple(place[s, :4]) == (X, y, mirror, t), s
        assert place[s, 5] == 2 and place[s, 4] == 1 and place[s, 6] == kt


def test_three_rows_downscaled_by_hand():
    """Nine boxes 100 texels wide and 130 down to 122 tall, in a 301 x 400
    atlas with 1-px gutters (W' = 303): at S = 1024 their padded widths are
    102, the prefix 0, 102, ..., 816 puts three boxes in each of rows 0, 1,
    2 (floor(P / 303)), and each row overflows (306 > 303).  At k the padded
    width is ceil(100 k / 1024) + 2, so three fit iff ceil(100 k / 1024) <=
    99, i.e. k <= 1013 (within 14 of S): k' = 1013, padded widths 101,
    padded heights ceil(h 1013 / 1024) + 2 = 131, 130, ..., 123.  Row 0 runs
    left to right at x = 0, 101, 202; rows 1 and 2 run right to left at
    x = 202, 101, 0 and drop onto the skyline: row 1 lands at 129, 130, 131
    and levels it at 257, row 2 lands at 257 and tops out at 382.  The next
    candidate, 1008, cannot beat a weighted scale of 1013, so the search
    stops there.  In a 300-wide atlas the rows overflow by 4 and fit only
    from k = 1003 down: too far below 1024, no tail is taken."""
    sizes = [(100, h) for h in range(130, 121, -1)]
    cs = synth.rectangles(sizes, 301, 400)
    params = oracle.default_params(topt=1000, hybrid_min=0)
    rec = oracle.prep(cs, params)
    perm = oracle.sort(rec)
    assert list(perm) == list(range(9)) and not rec[:, R["ROT"]].any()
    ok, place, stats = oracle.pack_scale(rec, perm, 301, 400, 1024, params)
    assert ok and stats[6] == 1013 and stats[5] == 3 and stats[3] == 382
    assert list(place[:, 3]) == [0, 0, 0, 1, 1, 1, 2, 2, 2]
    assert list(place[:, 2]) == [0, 0, 0, 1, 1, 1, 1, 1, 1]
    assert list(place[:, 0]) == [0, 101, 202, 202, 101, 0, 202, 101, 0]
    assert list(place[:, 1]) == [0, 0, 0, 129, 130, 131, 257, 257, 257]
    assert list(place[:, 6]) == [1013] * 9
    ok2, _, st2 = oracle.pack_scale(rec, perm, 301, 400, 1008, params)
    assert ok2 and st2[6] == 1008  # rows of 3 x 101 fit at 1008 itself
    r = oracle.pack(cs, params, all_scales=False)
    assert r.status == 0 and r.k == 1024 and list(r.place[:, 10]) == [1013] * 9
    assert r.score == 1013 * sum(_area2(sizes))
    narrow = synth.rectangles(sizes, 300, 400)
    rec = oracle.prep(narrow, params)
    ok3, pl3, st3 = oracle.pack_scale(rec, oracle.sort(rec), 300, 400, 1024, params)
    assert st3[6] == 0 and st3[5] == 0 and st3[7] == 9 and not np.any(pl3[:, 5] == 2)


@pytest.mark.parametrize("case", range(len(BOXES)))
def test_boxes_search_matches_brute_force(case):
    """The search keeps the successful candidate with the largest
    area-weighted scale, ties to the larger candidate (Sec. 4.4)."""
    sizes, W, H = BOXES[case]
    cs = synth.rectangles(sizes, W, H)
    params = oracle.default_params(topt=1000, hybrid_min=0)
    r = oracle.pack(cs, params, all_scales=True)
    area = sum(_area2(sizes))
    best, best_score, tails = 0, -1, 0
    rec = oracle.prep(cs, params)
    perm = oracle.sort(rec)
    for j in range(64, 0, -1):
        ok, kt, _ = skyline_tail(sizes, W, H, 16 * j)
        if ok is None:  # no tail taken: the oracle's own row-by-row result, every box at S
            ok, kt = oracle.pack_scale(rec, perm, W, H, 16 * j, params)[0], 16 * j
        else:
            tails += 1
        assert bool(r.success[j - 1]) == ok, j
        if ok and kt * area > best_score:
            best, best_score = 16 * j, kt * area
    assert tails > 10 or case < 3
    assert r.k == best and r.score == best_score
    assert r.status == 0 and np.all(r.place[:, 10] == best_score // area)


def _tall_then_small():
    rng = np.random.default_rng(5)
    sizes = [(int(rng.integers(32, 120)), int(h)) for h in np.linspace(240, 80, 12).astype(int)]
    sizes += [(int(rng.integers(4, 32)), int(rng.integers(8, 48))) for _ in range(300)]
    return sizes


def test_switch_point():
    """Sec. 4.4: sequential rows until no knee is live and the row's first
    (tallest) chart is below t_opt of the atlas height; tail rows after --
    where a tail scale within one grid step fits them, else the rows simply
    continue one by one (no row is folded by the prefix sum)."""
    sizes = _tall_then_small()
    W = H = 640
    cs = synth.rectangles(sizes, W, H)
    params = oracle.default_params(topt=50, hybrid_min=0)
    rec = oracle.prep(cs, params)
    perm = oracle.sort(rec)
    taken = 0
    for k in range(512, 1025, 32):
        ok, place, stats = oracle.pack_scale(rec, perm, W, H, k, params)
        placed = int(stats[4])
        assert stats[2] == 0  # no knees in this set (drops below 10 % of H)
        rows = place[:placed, 3]
        firsts = [int(np.argmax(rows == r)) for r in range(int(stats[0]))]
        h = [_ceil_div(int(rec[perm[s], R["HQ"]]) * k, 1 << 18) for s in firsts]
        below = [1000 * hh < 50 * H for hh in h]
        tail_rows = [bool(place[s, 5] == 2) for s in firsts]
        if stats[6] == 0:  # no tail scale fitted: every row folded one by one
            assert not any(tail_rows) and stats[5] == 0 and stats[7] == cs.n
            continue
        taken += 1
        first_tail = below.index(True) if True in below else len(below)
        assert tail_rows == [r >= first_tail for r in range(len(firsts))]
        assert stats[5] == len(firsts) - first_tail
        assert stats[5] > 0 and first_tail > 0
        assert stats[7] == firsts[first_tail]
        # the head keeps the candidate scale, the tail its own, within a step
        assert np.all(place[:firsts[first_tail], 6] == k)
        assert np.all(place[firsts[first_tail]:placed, 6] == stats[6]) and k - 14 <= stats[6] <= k
        # FastAtlas's alternation: one left-to-right row, then two right-to-left
        mirrors = [int(place[s, 2]) for s in firsts[first_tail:]]
        assert mirrors == [int(t % 3 != 0) for t in range(len(mirrors))]
    assert taken >= 2


def test_compacted_rows_are_tight_at_the_tail_scale():
    """In a left-to-right tail row each chart sits at the compacting distance
    (at the tail's scale k') from its predecessor, unless the clamp (chart
    s+1 never left of chart s-1's right edge) binds, in which case it
    touches that right edge; each row starts at the atlas's left edge."""
    cs = synth.stars(17, 2000, 1024)
    params = oracle.default_params(topt=50, hybrid_min=0)
    rec = oracle.prep(cs, params)
    perm = oracle.sort(rec)
    k = 448
    ok, place, stats = oracle.pack_scale(rec, perm, cs.atlas_w, cs.atlas_h, k, params)
    kt = int(stats[6])
    assert 0 < kt <= k
    d, _, _, wp, _ = oracle.scale_pairs(rec, perm, kt, params)
    placed = int(stats[4])
    checked = starts = 0
    for s in range(int(stats[7]), placed):
        if place[s, 2] != 0:
            continue
        if s == stats[7] or place[s - 1, 3] != place[s, 3]:
            assert place[s, 0] == 0
            starts += 1
        if s + 1 >= placed or place[s, 3] != place[s + 1, 3]:
            continue
        gap_ok = place[s + 1, 0] - place[s, 0] == wp[s] - d[s]
        clamp = place[s - 1, 3] == place[s, 3] and place[s + 1, 0] == place[s - 1, 0] + wp[s - 1]
        assert gap_ok or clamp, s
        assert place[s + 1, 0] - place[s, 0] >= wp[s] - d[s]
        checked += 1
    assert checked > 50 and starts > 2


def test_rows_follow_the_prefix_modulo_the_width():
    """The tail's rows are the prefix fold at the candidate scale cut modulo
    W' (each row's last chart may overflow it), recomputed here from the
    oracle's own widths and distances at S; every row fits W' at k'."""
    cs = synth.stars(19, 3000, 2048)
    params = oracle.default_params(topt=50, hybrid_min=0)
    rec = oracle.prep(cs, params)
    perm = oracle.sort(rec)
    S = 480
    ok, place, stats = oracle.pack_scale(rec, perm, cs.atlas_w, cs.atlas_h, S, params)
    c0, placed = int(stats[7]), int(stats[4])
    d, _, _, wp, _ = oracle.scale_pairs(rec, perm, S, params)
    P = [0]
    for s in range(c0, cs.n - 1):
        nx = P[-1] + wp[s] - d[s]
        if len(P) >= 2:
            nx = max(nx, P[-2] + wp[s - 1])
        P.append(nx)
    Wp = cs.atlas_w + 2
    rows = _rows_modulo(P, Wp)
    overflowing = sum(P[row[-1]] + wp[c0 + row[-1]] > (P[row[0]] // Wp + 1) * Wp for row in rows)
    assert overflowing > 0
    got = place[c0:placed, 3] - place[c0, 3]
    want = np.concatenate([[t] * len(row) for t, row in enumerate(rows)])[:placed - c0]
    assert np.array_equal(got, want)
    _, _, _, wpt, _ = oracle.scale_pairs(rec, perm, int(stats[6]), params)
    for row in rows[:int(stats[5])]:
        xs = [c0 + t for t in row]
        lo = min(place[s, 0] for s in xs)
        hi = max(place[s, 0] + wpt[s] for s in xs)
        assert lo >= 0 and hi <= Wp


@pytest.mark.parametrize("make", [lambda: synth.stars(17, 2000, 1024), lambda: synth.knees(3, 1500, 1024),
                                  lambda: synth.pareto20k(seed=4, n=2000, atlas=1024)])
@pytest.mark.parametrize("flags", [oracle.F_ALL, oracle.F_ALL & ~oracle.F_HC])
def test_invariants_with_the_tail(make, flags):
    """Overlap-free, gutters respected, inside the atlas, the candidate
    with the largest area-weighted scale returned -- with most rows folded
    by the prefix and drawn at the tail's own scale."""
    cs = make()
    params = oracle.default_params(topt=50, hybrid_min=0, flags=flags)
    r = oracle.pack(cs, params, all_scales=True)
    assert r.status == 0
    assert r.stats[5] > 0
    rec = oracle.prep(cs, params)
    res = check_packing(cs, r.place[:, 10], r.place, envelope_fn=lambda c, kc: oracle.envelope(rec[c], kc, params))
    assert res == dict(out_of_atlas=0, gutter_overlap=0, overlap=0, outside_envelope=0)
    j = r.k // 16
    assert r.success[j - 1] == 1
    # every larger successful candidate has a smaller area-weighted scale
    perm = oracle.sort(rec)
    area = np.array([_loop_area2(cs.polygon(perm[s])) for s in range(cs.n)], dtype=object)
    for jj in range(j + 1, 65):
        if r.success[jj - 1]:
            ok, pl, st = oracle.pack_scale(rec, perm, cs.atlas_w, cs.atlas_h, 16 * jj, params)
            assert ok and int(np.dot(area, pl[:, 6].astype(object))) < r.score


def test_small_atlases_keep_sequential_folding():
    """The tail applies only above hybrid_min charts (the paper: 10,000);
    at or below it the result is that of t_opt = 0."""
    cs = synth.stars(17, 2000, 1024)
    a = oracle.pack(cs, oracle.default_params(topt=50, hybrid_min=2000))
    b = oracle.pack(cs, oracle.default_params(topt=0))
    c = oracle.pack(cs, oracle.default_params(topt=50, hybrid_min=1999))
    assert a.k == b.k and np.array_equal(a.place, b.place) and a.stats[5] == 0
    assert c.stats[5] > 0


def _loop_area2(poly):
    """Twice the area of a vertex loop (shoelace magnitude), exact."""
    p = [(int(a), int(b)) for a, b in np.asarray(poly).reshape(-1, 2)]
    return abs(sum(x0 * y1 - x1 * y0 for (x0, y0), (x1, y1) in zip(p, p[1:] + p[:1])))


def test_paper_default_is_one_percent_above_ten_thousand():
    p = oracle.default_params()
    assert (p[7], p[8]) == (10, 10000)


def test_tail_clamp_keeps_non_neighbours_apart():
    """The compacted prefix keeps Algorithm 4's added rule: two small
    diamonds nest into a tall diamond's empty corner, and the third chart's
    compacted offset would reach into the first chart's columns, so it is
    clamped to the first chart's right edge (the pairwise interlock covers
    neighbours only)."""
    from test_oracle_pins import _diamond
    cs = synth.from_polygons([_diamond(60, 100), _diamond(10, 20), _diamond(10, 10)], 150, 300)
    params = oracle.default_params(topt=1000, hybrid_min=0)
    rec = oracle.prep(cs, params)
    perm = oracle.sort(rec)
    d, _, _, wp, _ = oracle.scale_pairs(rec, perm, 1024, params)
    ok, pl, st = oracle.pack_scale(rec, perm, 150, 300, 1024, params)
    assert ok and st[5] == 1 and list(pl[:, 3]) == [0, 0, 0] and list(pl[:, 5]) == [2, 2, 2]
    x = pl[:, 0]
    assert x[1] == wp[0] - d[0] < wp[0]
    assert x[1] + wp[1] - d[1] < x[0] + wp[0]
    assert x[2] == x[0] + wp[0]
