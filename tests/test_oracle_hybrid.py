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


def skyline_tail(sizes, W, H, k, g=1):
    """Independent brute force for boxes folded entirely by the tail: sorted
    by height, padded sizes at scale k, prefix offsets = padded widths,
    rows broken at multiples of L = W' - wmax + 1, FastAtlas directions, each
    box dropped onto the skyline.  Returns (success, {sorted pos: (X, y,
    mirror, tail row)})."""
    order = sorted(range(len(sizes)), key=lambda i: -sizes[i][1])  # stable
    Wp, Hp = W + 2 * g, H + 2 * g
    wp = [_ceil_div(sizes[i][0] * k, 1024) + 2 * g for i in order]
    hp = [_ceil_div(sizes[i][1] * k, 1024) + 2 * g for i in order]
    if max(wp) > Wp:
        return False, {}
    L = Wp - max(wp) + 1
    P = np.concatenate([[0], np.cumsum(wp)[:-1]])
    groups = {}
    for s, p in enumerate(P):
        groups.setdefault(int(p) // L, []).append(s)
    front = np.zeros(Wp, np.int64)
    out = {}
    for t, r in enumerate(sorted(groups)):
        mirror = t % 3 != 0
        ys = {}
        for s in groups[r]:
            x = int(P[s]) - r * L
            X = Wp - x - wp[s] if mirror else x
            ys[s] = (X, int(front[X:X + wp[s]].max()))
        for s, (X, y) in ys.items():
            front[X:X + wp[s]] = np.maximum(front[X:X + wp[s]], y + hp[s])
            out[s] = (X, y, int(mirror), t)
        if front.max() > Hp:
            return False, out
    return True, out


BOXES = [[(3, 5), (2, 2), (4, 6), (1, 3), (5, 5), (2, 4), (3, 3), (1, 1), (2, 6), (4, 4)] * 3,
         [(1, 2), (2, 3), (3, 3), (1, 1)] * 9 + [(6, 7), (5, 8)]]


@pytest.mark.parametrize("case", range(len(BOXES)))
@pytest.mark.parametrize("k", [256, 512, 768, 1024])
@pytest.mark.parametrize("g", [1, 0, 2])
def test_boxes_match_skyline_brute_force(case, k, g):
    sizes = BOXES[case]
    W, H = 17, 40
    cs = synth.rectangles(sizes, W, H)
    params = oracle.default_params(topt=1000, hybrid_min=0, gutter=g)  # every row is a tail row
    rec = oracle.prep(cs, params)
    perm = oracle.sort(rec)
    ok, place, stats = oracle.pack_scale(rec, perm, W, H, k, params)
    bok, exp = skyline_tail(sizes, W, H, k, g)
    assert ok == bok
    placed = int(stats[4])
    assert stats[5] == stats[0]  # all rows are tail rows
    for s in range(placed):
        X, y, mirror, t = exp[s]
        assert tuple(place[s, :4]) == (X, y, mirror, t), s
        assert place[s, 5] == 2 and place[s, 4] == 1


def test_boxes_search_matches_brute_force():
    sizes = BOXES[0]
    W, H = 17, 40
    cs = synth.rectangles(sizes, W, H)
    params = oracle.default_params(topt=1000, hybrid_min=0)
    r = oracle.pack(cs, params, all_scales=True)
    for j in range(1, 65):
        assert bool(r.success[j - 1]) == skyline_tail(sizes, W, H, 16 * j)[0], j
    best = max(16 * j for j in range(1, 65) if skyline_tail(sizes, W, H, 16 * j)[0])
    assert r.k == best


def _tall_then_small():
    rng = np.random.default_rng(5)
    sizes = [(int(rng.integers(8, 30)), int(h)) for h in np.linspace(60, 20, 12).astype(int)]
    sizes += [(int(rng.integers(1, 8)), int(rng.integers(2, 12))) for _ in range(300)]
    return sizes


def test_switch_point():
    """Sec. 4.4: sequential rows until no knee is live and the row's first
    (tallest) chart is below t_opt of the atlas height; tail rows after."""
    sizes = _tall_then_small()
    W = H = 160
    cs = synth.rectangles(sizes, W, H)
    params = oracle.default_params(topt=50, hybrid_min=0)
    rec = oracle.prep(cs, params)
    perm = oracle.sort(rec)
    for k in (512, 768, 1024):
        ok, place, stats = oracle.pack_scale(rec, perm, W, H, k, params)
        placed = int(stats[4])
        assert stats[2] == 0  # no knees in this set (drops below 10 % of H)
        rows = place[:placed, 3]
        firsts = [int(np.argmax(rows == r)) for r in range(int(stats[0]))]
        h = [_ceil_div(int(rec[perm[s], R["HQ"]]) * k, 1 << 18) for s in firsts]
        below = [1000 * hh < 50 * H for hh in h]
        tail_rows = [bool(place[s, 5] == 2) for s in firsts]
        first_tail = below.index(True) if True in below else len(below)
        assert tail_rows == [r >= first_tail for r in range(len(firsts))]
        assert stats[5] == len(firsts) - first_tail
        assert stats[5] > 0 and first_tail > 0
        # FastAtlas's alternation: one left-to-right row, then two right-to-left
        mirrors = [int(place[s, 2]) for s in firsts[first_tail:]]
        assert mirrors == [int(t % 3 != 0) for t in range(len(mirrors))]


def test_compacted_prefix_is_tight():
    """In a left-to-right tail row each chart sits at the compacting distance
    from its predecessor, unless the clamp (chart s+1 never left of chart
    s-1's right edge) binds, in which case it touches that right edge."""
    cs = synth.stars(17, 400, 512)
    params = oracle.default_params(topt=200, hybrid_min=0)
    rec = oracle.prep(cs, params)
    perm = oracle.sort(rec)
    k = 448
    ok, place, stats = oracle.pack_scale(rec, perm, cs.atlas_w, cs.atlas_h, k, params)
    d, _, _, wp, _ = oracle.scale_pairs(rec, perm, k, params)
    placed = int(stats[4])
    checked = 0
    for s in range(1, placed - 1):
        same = place[s, 3] == place[s + 1, 3] and place[s, 5] == 2
        if not same or place[s, 2] != 0:
            continue
        gap_ok = place[s + 1, 0] - place[s, 0] == wp[s] - d[s]
        clamp = place[s - 1, 3] == place[s, 3] and place[s + 1, 0] == place[s - 1, 0] + wp[s - 1]
        assert gap_ok or clamp, s
        assert place[s + 1, 0] - place[s, 0] >= wp[s] - d[s]
        checked += 1
    assert checked > 50


@pytest.mark.parametrize("make", [lambda: synth.stars(23, 600, 512), lambda: synth.knees(3, 500, 1024),
                                  lambda: synth.pareto20k(seed=4, n=1200, atlas=1024)])
@pytest.mark.parametrize("flags", [oracle.F_ALL, oracle.F_ALL & ~oracle.F_HC])
def test_invariants_with_the_tail(make, flags):
    """Overlap-free, gutters respected, inside the atlas, the largest
    successful candidate returned -- with most rows folded by the prefix."""
    cs = make()
    params = oracle.default_params(topt=100, hybrid_min=0, flags=flags)
    r = oracle.pack(cs, params, all_scales=True)
    assert r.status == 0
    assert r.stats[5] > 0
    rec = oracle.prep(cs, params)
    res = check_packing(cs, r.k, r.place, envelope_fn=lambda c: oracle.envelope(rec[c], r.k, params))
    assert res == dict(out_of_atlas=0, gutter_overlap=0, overlap=0, outside_envelope=0)
    j = r.k // 16
    assert r.success[j - 1] == 1 and not np.any(r.success[j:])


def test_small_atlases_keep_sequential_folding():
    """The tail applies only above hybrid_min charts (the paper: 10,000);
    at or below it the result is that of t_opt = 0."""
    cs = synth.stars(29, 300, 512)
    a = oracle.pack(cs, oracle.default_params(topt=100, hybrid_min=300))
    b = oracle.pack(cs, oracle.default_params(topt=0))
    c = oracle.pack(cs, oracle.default_params(topt=100, hybrid_min=299))
    assert a.k == b.k and np.array_equal(a.place, b.place) and a.stats[5] == 0
    assert c.stats[5] > 0


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
