"""GPU tests of the overlap and gutter counter (tabi_check_packing_device
and the serving loop's check behind every batch): the paper's overlap
metric (App. B) counted on the device equals the CPU count of
tests/exact_cover.py -- zero on packings, and the exact counts on
placements made to overlap, to break the gutter and to leave the atlas."""
from __future__ import annotations

import numpy as np
import pytest

import synth
from exact_cover import check_packing

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # the -m gpu suite runs on a GPU machine only
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_2602_07782_gb300 import tabi  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = tabi.Context(arena_bytes=1 << 30)
    yield c
    c.close()


def _dev(cs, place):
    dev = torch.device("cuda:0")
    offs = torch.from_numpy(cs.offsets.view(np.int32).copy()).to(dev)
    verts = torch.from_numpy(cs.verts.copy()).to(dev)
    pl = torch.from_numpy(np.ascontiguousarray(place).view(np.uint8).copy()).to(dev)
    return offs, verts, pl


def _cpu_counts(cs, place, g):
    arr = np.stack([place[f].astype(np.int64) for f in ("x", "y", "rot90", "flip_x", "flip_y", "mirror")], 1)
    r = check_packing(cs, place["k"].astype(np.int64), arr, gutter=g)
    return r["overlap"], r["gutter_overlap"], r["out_of_atlas"]


def _gpu_counts(ctx, cs, place, g):
    offs, verts, pl = _dev(cs, place)
    st, q = ctx.check_packing_device(cs.atlas_w, cs.atlas_h, g, cs.n, cs.nv, offs, verts, pl)
    assert st == tabi.TABI_OK, ctx.last_error()
    return q


@pytest.mark.parametrize("make,params", [
    (lambda: synth.stars(3, 300, 512), {}),
    (lambda: synth.knees(2, 250, 1024), {}),
    (lambda: synth.stars(17, 2000, 1024), {"topt_permille": 50, "hybrid_min_charts": 0}),  # tail charts at k'
    (lambda: synth.stars(6, 200, 512), {"gutter": 3}),
    (lambda: synth.plain64(seed=2), {"gutter": 0}),
])
def test_packings_count_zero_like_the_cpu(ctx, make, params):
    cs = make()
    p = tabi.params_default(**params)
    res = ctx.pack(cs, p)
    assert res.status == tabi.TABI_OK, ctx.last_error()
    g = p.gutter
    assert _gpu_counts(ctx, cs, res.place, g) == (0, 0, 0)
    assert _cpu_counts(cs, res.place, g) == (0, 0, 0)


@pytest.mark.parametrize("g", [1, 2, 0])
def test_broken_placements_match_the_cpu_count(ctx, g):
    """Placements moved on the host: a chart dropped onto another, one moved
    next to a neighbour inside the gutter, one pushed partly out of the
    atlas, one mirrored and rotated differently -- the device counts equal
    the CPU counts exactly."""
    cs = synth.stars(9, 120, 512)
    res = ctx.pack(cs, tabi.params_default(gutter=g))
    assert res.status == tabi.TABI_OK
    rng = np.random.default_rng(g + 5)
    for trial in range(4):
        pl = res.place.copy()
        idx = rng.choice(cs.n, 6, replace=False)
        pl["x"][idx[0]] = pl["x"][idx[1]] + int(rng.integers(-3, 4))      # onto another chart
        pl["y"][idx[0]] = pl["y"][idx[1]] + int(rng.integers(-3, 4))
        pl["x"][idx[2]] += int(rng.integers(1, 3))                        # a nudge: gutter contact
        pl["x"][idx[3]] = cs.atlas_w - 3                                  # partly outside
        pl["y"][idx[4]] = -2
        pl["mirror"][idx[5]] ^= 1
        pl["k"][idx[5]] = max(16, int(pl["k"][idx[5]]) - 50)            # its own (smaller) scale
        want = _cpu_counts(cs, pl, g)
        got = _gpu_counts(ctx, cs, pl, g)
        assert got == want, (trial, got, want)
        assert want[0] > 0 and want[2] > 0


def test_large_charts_and_many_vertices(ctx):
    """Charts with more vertices than a warp keeps in shared memory, and
    charts wider than a warp's column chunk (several warps per chart)."""
    rng = np.random.default_rng(3)
    polys = []
    for i in range(6):
        m = 200 + 40 * i
        ang = np.sort(rng.uniform(0, 2 * np.pi, m))
        r = rng.uniform(0.6, 1.0, m) * (60 + 30 * i) * 256
        polys.append([(int(256 * 200 + a * np.cos(t)), int(256 * 200 + a * np.sin(t))) for t, a in zip(ang, r)])
    cs = synth.from_polygons(polys, 700, 700)
    res = ctx.pack(cs, tabi.params_default())
    assert res.status == tabi.TABI_OK
    pl = res.place.copy()
    assert _gpu_counts(ctx, cs, pl, 1) == _cpu_counts(cs, pl, 1) == (0, 0, 0)
    pl["x"][1] = pl["x"][0] + 7
    pl["y"][1] = pl["y"][0] + 5
    assert _gpu_counts(ctx, cs, pl, 1) == _cpu_counts(cs, pl, 1)


def test_served_results_carry_zero_counts():
    sets = [synth.stars(40 + i, n, side) for i, (n, side) in enumerate([(50, 256), (400, 512), (1500, 1024)])]
    srv = tabi.Server(lanes=2, max_batch=8, arena_bytes=1 << 30)
    try:
        tickets = [srv.submit(cs)[1] for cs in sets * 3]
        for t in tickets:
            st, r = srv.wait(t)
            assert st == tabi.TABI_OK and r.status == tabi.TABI_OK
            assert (r.overlap_texels, r.gutter_texels, r.outside_texels) == (0, 0, 0)
        s = srv.stats()
        assert s["checked"] == len(tickets) and s["check_violations"] == 0 and s["check_ns"] > 0
    finally:
        srv.close()
