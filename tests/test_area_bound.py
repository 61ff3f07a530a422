"""The area bound on the candidate scales (CPU, against the oracle).

Placed charts never overlap and lie inside the atlas (Sec. 5 packs without
overlap; the envelopes are conservative covers), so a candidate k can only
succeed if the summed polygon area at scale k/1024 is at most W * H.  The
GPU path skips the candidates above that bound.  These tests check, with
the oracle, that every skipped candidate indeed fails and that the chosen
scale is never above the bound.
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


def top_candidate(cs) -> int:
    """Largest j with area2 * k^2 <= W H 2^37 (k = 16 (j + 1)); -1 if none."""
    s2 = twice_area_q8(cs)
    lim = cs.atlas_w * cs.atlas_h << 37
    jt = -1
    for j in range(64):
        k = 16 * (j + 1)
        if s2 * k * k <= lim:
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
    """64 squares of 8x8 texels tile a 64x64 atlas exactly at k = 1024 with
    no gutter; the bound allows k = 1024 and nothing less is forced."""
    cs = synth.rectangles([(8, 8)] * 64, 64, 64)
    assert top_candidate(cs) == 63
    cs2 = synth.rectangles([(8, 8)] * 65, 64, 64)
    assert top_candidate(cs2) == 62  # (k/1024)^2 * 65 * 64 <= 4096  <=>  k <= 1016
