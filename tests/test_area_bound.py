"""The area bound on the candidate scales (CPU, against the oracle).

Placed charts never overlap (Sec. 5: gutters of g texels between charts;
the envelopes are conservative covers): the covers dilated by g are
disjoint inside the padded atlas (W + 2g) x (H + 2g), so a candidate k can
only succeed if the charts' dilated areas at scale k/1024 sum to at most
that.  The GPU path skips the candidates above the bound.  These tests
check, with the oracle, that every skipped candidate indeed fails and that
the chosen scale is never above the bound, and the dilation lemma itself.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth


def twice_area_q8(cs) -> int:
    """Twice the summed polygon area in Q.8^2 units (exact shoelace)."""
    total = 0
    for i in range(cs.n):
        p = cs.polygon(i).astype(object)
        x, y = p[:, 0], p[:, 1]
        total += abs(int(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y)))
    return total


def larger_extents_q8(cs) -> int:
    """Summed larger AABB side of the charts (Q.8)."""
    total = 0
    for i in range(cs.n):
        p = cs.polygon(i).astype(np.int64)
        ext = p.max(axis=0) - p.min(axis=0)
        total += int(ext.max())
    return total


def top_candidate(cs, gutter: int = 1) -> int:
    """Largest j (k = 16 (j + 1)) whose dilated-area bound holds; -1 if none.
    The covers dilated by g are disjoint inside (W + 2g) x (H + 2g), and a
    connected polygon of area A and larger extent E dilated by g covers at
    least A + 2 g E + 4 g^2 (texels, at scale k/1024)."""
    s2 = twice_area_q8(cs)
    ext = larger_extents_q8(cs)
    g = gutter
    lim = ((cs.atlas_w + 2 * g) * (cs.atlas_h + 2 * g)) << 37
    jt = -1
    for j in range(64):
        k = 16 * (j + 1)
        if s2 * k * k + ((2 * g * k * ext) << 19) + ((4 * g * g * cs.n) << 37) <= lim:
            jt = j
    return jt


CASES = {
    "plain64": lambda: synth.plain64(seed=1),
    "stars200": lambda: synth.stars(3, 200, 512),
    "knees150": lambda: synth.knees(5, 150, 512),
    "dense": lambda: synth.stars(4, 120, 256, density=12.0),
    "squares": lambda: synth.rectangles([(8, 8)] * 64, 64, 64),
}


@pytest.mark.parametrize("name", list(CASES))
def test_candidates_above_the_area_bound_fail(name):
    cs = CASES[name]()
    jt = top_candidate(cs)
    rec = oracle.prep(cs)
    perm = oracle.sort(rec)
    r = oracle.pack(cs)
    assert r.status != 0 or r.k <= 16 * (jt + 1)
    for j in range(jt + 1, min(64, jt + 4)):
        ok, _, _ = oracle.pack_scale(rec, perm, cs.atlas_w, cs.atlas_h, 16 * (j + 1))
        assert not ok, j


def test_area_bound_is_tight_for_exact_tiling():
    """Without a gutter the bound is the plain area bound: 64 squares of 8x8
    texels tile a 64x64 atlas exactly at k = 1024; 65 do not fit above
    k = 1016.  With gutter 1 a square of side 8x dilates to at least
    64x^2 + 16x + 4 texels (x = k/1024), and 64 of them must fit 66 x 66."""
    cs = synth.rectangles([(8, 8)] * 64, 64, 64)
    assert top_candidate(cs, gutter=0) == 63
    cs2 = synth.rectangles([(8, 8)] * 65, 64, 64)
    assert top_candidate(cs2, gutter=0) == 62  # (k/1024)^2 * 65 * 64 <= 4096  <=>  k <= 1016
    # gutter 1: 64 (64 x^2 + 16 x + 4) <= 66^2  <=>  x <= 0.8833  <=>  k <= 904.5
    assert top_candidate(cs, gutter=1) == 55  # k = 896


def test_dilation_lemma_on_rasterised_polygons():
    """The dilated area of a connected polygon is at least A + 2 g E + 4 g^2:
    checked on fine rasterisations of the workload's chart shapes."""
    cs = synth.plain64(seed=3)
    g = 1.0
    for i in range(0, cs.n, 8):
        p = cs.polygon(i).astype(np.float64) / 256.0
        p -= p.min(axis=0)
        w, h = p.max(axis=0)
        step = 0.05
        xs = np.arange(-g, w + g, step) + step / 2
        ys = np.arange(-g, h + g, step) + step / 2
        X, Y = np.meshgrid(xs, ys)
        inside = _points_in_polygon(X.ravel(), Y.ravel(), p).reshape(X.shape)
        # dilate by g with a square structuring element on the fine grid
        r = int(round(g / step))
        from scipy.ndimage import binary_dilation
        dil = binary_dilation(inside, structure=np.ones((2 * r + 1, 2 * r + 1), bool))
        area_dil = dil.sum() * step * step
        area = 0.5 * abs(np.sum(p[:, 0] * np.roll(p[:, 1], -1) - np.roll(p[:, 0], -1) * p[:, 1]))
        assert area_dil >= area + 2 * g * max(w, h) + 4 * g * g - 0.5  # grid error margin


def _points_in_polygon(x, y, poly):
    inside = np.zeros(x.shape, bool)
    n = len(poly)
    for a in range(n):
        x0, y0 = poly[a]
        x1, y1 = poly[(a + 1) % n]
        cond = (y0 > y) != (y1 > y)
        with np.errstate(divide="ignore", invalid="ignore"):
            xc = x0 + (y - y0) * (x1 - x0) / (y1 - y0)
        inside ^= cond & (x < xc)
    return inside
