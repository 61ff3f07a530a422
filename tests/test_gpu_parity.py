"""GPU parity: every step of the CUDA path against the CPU oracle, bit for
bit, through the C ABI (include/tabi.h) and its Python binding.

Integer path: the bar is exact equality of every chart record, permutation,
envelope, compacting distance, interlock flag, per-scale success and
placement, and the final scale and placements.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # the -m gpu suite runs on a GPU machine only
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_2602_07782_gb300 import tabi  # noqa: E402

R = oracle.R
K = oracle.K


@pytest.fixture(scope="module")
def ctx():
    c = tabi.Context(arena_bytes=3 << 30)
    yield c
    c.close()


def gpu_params(**kw):
    kw.setdefault("scale_fanout", 64)
    return tabi.params_default(**kw)


def oracle_params(p):
    # the oracle knows the method's flags only (TABI_F_EVAL_ALL is an inspection aid)
    return oracle.default_params(gutter=p.gutter, knee_abs=p.knee_abs_pct, knee_rel=p.knee_rel_pct,
                                 lr_sig=p.lr_sig_pct, knee_margin=p.knee_margin, flags=p.flags & tabi.F_ALL,
                                 laabb_k=p.laabb_count, topt=p.topt_permille, hybrid_min=p.hybrid_min_charts)


SMALL = {
    "plain64_s1": lambda: synth.plain64(seed=1),
    "plain64_s2": lambda: synth.plain64(seed=2),
    "stars300": lambda: synth.stars(3, 300, 512),
    "knees300": lambda: synth.knees(1, 300, 1024),
    "knees200_512": lambda: synth.knees(5, 200, 512),
    "strips": lambda: synth.pareto20k(seed=9, n=1500, atlas=1024),
}


def _check_prep(ctx, cs, op):
    info = ctx.charts()
    rec = oracle.prep(cs, op)
    nk = int(op[6])  # local AABBs per axis; record slot t holds slice t * nk // 10
    slot = np.arange(10) * nk // 10
    assert np.all(info["valid"] == 1)
    for f, col in (("Wq", "WQ"), ("Hq", "HQ"), ("rot90", "ROT"), ("flip_y", "FLIPY"),
                   ("flip_x", "FLIPX"), ("obb_m", "OBBM"), ("u0", "U0"), ("u1", "U1"),
                   ("v0", "V0"), ("v1", "V1"), ("area_top", "ATOP"), ("area_bot", "ABOT"),
                   ("area_left", "ALEFT"), ("area_right", "ARIGHT"), ("area_bl2", "ABL2"),
                   ("area_br2", "ABR2")):
        assert np.array_equal(info[f].astype(np.int64), rec[:, R[col]]), f
    for f, col in (("ylo", "YLO"), ("yhi", "YHI"), ("xlo", "XLO"), ("xhi", "XHI")):
        assert np.array_equal(info[f].astype(np.int64), rec[:, R[col] + slot]), f
    perm = ctx.perm()
    assert np.array_equal(perm, oracle.sort(rec))
    return rec, perm


def test_prep_group_widths(ctx):
    """Prep runs 32, 16, 8 or 4 lanes per chart, by the chart count against
    the multiprocessors' resident warps; every width gives the oracle's
    chart records and sorted order."""
    warps = 16 * torch.cuda.get_device_properties(0).multi_processor_count
    seen = set()
    for i, n in enumerate([warps // 2, warps * 3 // 2, warps * 3, warps * 5]):
        cs = synth.stars(40 + i, n, 4096)
        p = gpu_params()
        ctx.pack(cs, p)
        seen.add(ctx.prep_group())
        _check_prep(ctx, cs, oracle_params(p))
    assert seen == {32, 16, 8, 4}


@pytest.mark.parametrize("name", list(SMALL))
@pytest.mark.parametrize("topt", [0, 60])
def test_steps_parity(ctx, name, topt):
    """prep, sort, envelopes, distances/flags and every candidate's row loop
    (topt 60: rows past 6 % of the atlas height folded by the prefix sum of
    Sec. 4.4, whatever the chart count)."""
    cs = SMALL[name]()
    p = gpu_params(flags=tabi.F_ALL | tabi.F_EVAL_ALL,  # every candidate runs to its end
                   topt_permille=topt, hybrid_min_charts=0)
    op = oracle_params(p)
    res = ctx.pack(cs, p)
    assert res.status == tabi.TABI_OK, ctx.last_error()
    rec, perm = _check_prep(ctx, cs, op)
    for j in range(0, 64, 1 if cs.n <= 300 else 7):
        k = 16 * (j + 1)
        hdr, place = ctx.scale_result(j, cs.n)
        ok, opl, ost = oracle.pack_scale(rec, perm, cs.atlas_w, cs.atlas_h, k, op)
        assert hdr[0] == int(ok), j
        assert list(hdr[1:6]) == [ost[0], ost[1], ost[2], ost[3], ost[4]], j
        # Sec. 4.4: rows pushed by the tail, its scale k' and first chart
        assert [hdr[7], hdr[8], hdr[9]] == [ost[5], ost[6], ost[7]], j
        # the tail's charts are drawn (and compacted) at k' once it is found
        kt, c0 = int(ost[6]), int(ost[7])
        ks = [kt if (kt and s >= c0) else k for s in range(cs.n)]
        env = ctx.envelopes(j, cs.n)
        for s in range(cs.n):
            e = oracle.envelope_padded(rec[perm[s]], ks[s], op)
            wp, hp, top, bot, left, right, mb = env[s]
            assert (wp, hp) == (e.w, e.h), (j, s)
            assert np.array_equal(top, e.top) and np.array_equal(bot, e.bot), (j, s)
            assert np.array_equal(left, e.left) and np.array_equal(right, e.right), (j, s)
            assert mb == e.bot.max()
        d, ca, cb = ctx.pairs(j, cs.n)
        od, oca, ocb, owp, ohp = oracle.scale_pairs(rec, perm, k, op)
        lim = c0 if kt else cs.n - 1  # pairs at k; with a tail at k', those from the first tail chart on
        assert np.array_equal(d[:lim], od[:lim]), j
        assert np.array_equal(ca[:lim], oca[:lim]) and np.array_equal(cb[:lim], ocb[:lim]), j
        if kt:
            td, tca, tcb, _, _ = oracle.scale_pairs(rec, perm, kt, op)
            assert np.array_equal(d[c0:-1], td[c0:-1]), j
            assert np.array_equal(ca[c0:-1], tca[c0:-1]) and np.array_equal(cb[c0:-1], tcb[c0:-1]), j
        placed = int(ost[4])
        bits = opl[:placed, 2] | (opl[:placed, 4] << 1) | (opl[:placed, 5] << 2)
        assert np.array_equal(place[:placed, 0], opl[:placed, 0]), j
        assert np.array_equal(place[:placed, 1], opl[:placed, 1]), j
        assert np.array_equal(place[:placed, 2], opl[:placed, 3]), j
        assert np.array_equal(place[:placed, 3], bits), j


def _compare_pack(cs, res, op):
    o = oracle.pack(cs, op)
    assert res.status == {0: 0, 2: 2, 1: 1}[o.status]
    assert res.k == o.k
    if o.status == 0:
        pl = res.place
        assert np.array_equal(pl["x"], o.place[:, 0])
        assert np.array_equal(pl["y"], o.place[:, 1])
        assert np.array_equal(pl["rot90"], o.place[:, 2])
        assert np.array_equal(pl["flip_x"], o.place[:, 3])
        assert np.array_equal(pl["flip_y"], o.place[:, 4])
        assert np.array_equal(pl["mirror"], o.place[:, 5])
        assert np.array_equal(pl["k"], o.place[:, 10])  # each chart's scale (the tail's k')
    return o


@pytest.mark.parametrize("name", list(SMALL))
@pytest.mark.parametrize("fanout", [64, 8, 1])
def test_pack_parity(ctx, name, fanout):
    cs = SMALL[name]()
    p = gpu_params(scale_fanout=fanout)
    res = ctx.pack(cs, p)
    _compare_pack(cs, res, oracle_params(p))


@pytest.mark.parametrize("name,make", [("stars2k", synth.stars2k), ("pareto20k", synth.pareto20k)])
def test_full_size_parity(ctx, name, make):
    """The full-size workloads, in the launch configuration the benchmark
    times (scale_fanout 64), bit-exact against the oracle."""
    cs = make()
    p = gpu_params()
    res = ctx.pack(cs, p)
    assert res.status == 0, ctx.last_error()
    _compare_pack(cs, res, oracle_params(p))


@pytest.mark.parametrize("flags", [tabi.F_ALL & ~tabi.F_HC, tabi.F_ALL & ~tabi.F_BALANCE,
                                   tabi.F_HC | tabi.F_BALANCE, tabi.F_ALL & ~tabi.F_OBB,
                                   tabi.F_ALL & ~tabi.F_LAABB, 0])
def test_ablation_parity(ctx, flags):
    cs = synth.knees(2, 250, 1024)
    p = gpu_params(flags=flags)
    _compare_pack(cs, ctx.pack(cs, p), oracle_params(p))


@pytest.mark.parametrize("name", list(SMALL))
@pytest.mark.parametrize("fanout", [64, 8, 1])
@pytest.mark.parametrize("topt", [20, 150])
def test_tail_pack_parity(ctx, name, fanout, topt):
    """The prefix-sum tail (Sec. 4.4) in every candidate, whole packs."""
    cs = SMALL[name]()
    p = gpu_params(scale_fanout=fanout, topt_permille=topt, hybrid_min_charts=0)
    _compare_pack(cs, ctx.pack(cs, p), oracle_params(p))


@pytest.mark.parametrize("flags", [tabi.F_ALL & ~tabi.F_HC, tabi.F_ALL & ~tabi.F_BALANCE, 0])
def test_tail_ablation_parity(ctx, flags):
    cs = synth.knees(2, 250, 1024)
    p = gpu_params(flags=flags, topt_permille=100, hybrid_min_charts=0)
    _compare_pack(cs, ctx.pack(cs, p), oracle_params(p))


def test_tail_threshold_by_chart_count(ctx):
    """The tail applies above hybrid_min_charts only (the paper: 10,000)."""
    cs = synth.stars(17, 2000, 1024)
    for hmin in (1999, 2000):
        p = gpu_params(topt_permille=50, hybrid_min_charts=hmin)
        o = _compare_pack(cs, ctx.pack(cs, p), oracle_params(p))
        assert (o.stats[5] > 0) == (hmin < 2000)


@pytest.mark.parametrize("topt", [50, 150])
def test_tail_candidates_taken_and_abandoned(ctx, topt):
    """Every candidate of a 2,000-chart atlas with the tail from 5 % (15 %) of
    the atlas height: candidates whose rows fit within a grid step push the
    tail at its own scale, the others fold the rest row by row; each
    candidate's outcome, tail scale, first tail chart and placements, and the
    envelopes at the tail scale, against the oracle."""
    cs = synth.stars(17, 2000, 1024)
    p = gpu_params(flags=tabi.F_ALL | tabi.F_EVAL_ALL, topt_permille=topt, hybrid_min_charts=0)
    op = oracle_params(p)
    res = ctx.pack(cs, p)
    assert res.status == tabi.TABI_OK, ctx.last_error()
    rec = oracle.prep(cs, op)
    perm = oracle.sort(rec)
    taken = abandoned = 0
    for j in range(20, 40):
        k = 16 * (j + 1)
        hdr, place = ctx.scale_result(j, cs.n)
        ok, opl, ost = oracle.pack_scale(rec, perm, cs.atlas_w, cs.atlas_h, k, op)
        assert hdr[0] == int(ok) and list(hdr[1:6]) == [int(v) for v in ost[:5]], j
        assert [hdr[7], hdr[8], hdr[9]] == [int(ost[5]), int(ost[6]), int(ost[7])], j
        placed = int(ost[4])
        assert np.array_equal(place[:placed, 0], opl[:placed, 0]), j
        assert np.array_equal(place[:placed, 1], opl[:placed, 1]), j
        kt, c0 = int(ost[6]), int(ost[7])
        if kt:
            taken += 1
            env = ctx.envelopes(j, cs.n)
            for s in range(c0, cs.n, 37):
                e = oracle.envelope_padded(rec[perm[s]], kt, op)
                assert (env[s][0], env[s][1]) == (e.w, e.h) and np.array_equal(env[s][2], e.top), (j, s)
        elif ost[7] == cs.n and ok:
            abandoned += 1
    assert taken > 0
    _compare_pack(cs, res, op)


@pytest.mark.parametrize("count", [2, 5])
def test_laabb_count_parity(ctx, count):
    """Tab. 13's local-AABB counts: chart records, envelopes at a spread of
    candidates and the packing, each against the oracle at that count."""
    cs = synth.knees(8, 220, 1024)
    p = gpu_params(flags=tabi.F_ALL | tabi.F_EVAL_ALL, laabb_count=count)
    op = oracle_params(p)
    res = ctx.pack(cs, p)
    assert res.status == tabi.TABI_OK, ctx.last_error()
    rec, perm = _check_prep(ctx, cs, op)
    for j in (3, 20, 37, 63):
        env = ctx.envelopes(j, cs.n)
        for s in range(cs.n):
            e = oracle.envelope_padded(rec[perm[s]], 16 * (j + 1), op)
            wp, hp, top, bot, left, right, mb = env[s]
            assert (wp, hp) == (e.w, e.h), (j, s)
            assert np.array_equal(top, e.top) and np.array_equal(bot, e.bot), (j, s)
            assert np.array_equal(left, e.left) and np.array_equal(right, e.right), (j, s)
    _compare_pack(cs, res, op)
    for flags in (tabi.F_ALL & ~tabi.F_OBB, tabi.F_ALL):
        p = gpu_params(flags=flags, laabb_count=count, scale_fanout=8)
        _compare_pack(cs, ctx.pack(cs, p), oracle_params(p))


def test_laabb_count_rejected(ctx):
    cs = synth.stars(6, 20, 256)
    for count in (0, 1, 3, 11):
        assert ctx.pack(cs, gpu_params(laabb_count=count)).status == tabi.TABI_ERR_INVALID_ARG
    assert ctx.pack(cs, gpu_params()).status == tabi.TABI_OK


@pytest.mark.parametrize("gutter", [0, 2, 3])
def test_gutter_parity(ctx, gutter):
    cs = synth.stars(6, 200, 512)
    p = gpu_params(gutter=gutter)
    _compare_pack(cs, ctx.pack(cs, p), oracle_params(p))


def test_edge_cases(ctx):
    p = gpu_params()
    op = oracle_params(p)
    # a single chart
    cs = synth.stars(21, 1, 256, density=0.3)
    _compare_pack(cs, ctx.pack(cs, p), op)
    # equal squares (every direction ties)
    cs = synth.rectangles([(7, 7)] * 50, 100, 60)
    _compare_pack(cs, ctx.pack(cs, p), op)
    # a chart that fits at no candidate scale
    cs = synth.rectangles([(300, 300)], 2, 2)
    assert ctx.pack(cs, p).status == tabi.TABI_ERR_NO_FIT
    # non-square atlas, knees, ragged sizes
    cs = synth.knees(7, 123, 777)
    cs.atlas_h = 333
    _compare_pack(cs, ctx.pack(cs, p), op)
    # the nesting diamonds where the second-neighbour clamp binds
    def diamond(W, H):
        W, H = W * 256, H * 256
        return [(W // 2, 0), (W, H // 2), (W // 2, H), (0, H // 2)]
    cs = synth.from_polygons([diamond(60, 100), diamond(10, 20), diamond(10, 10)], 78, 300)
    _compare_pack(cs, ctx.pack(cs, p), op)


def _looped(poly, times):
    return [q for _ in range(times) for q in poly]


def test_self_overlapping_loops_keep_the_oracle_result(ctx):
    """Loops that wind twice or cross themselves have a shoelace area above
    the area they cover, so the area bounds (a shortcut the oracle does not
    take) must not count it: such loops enter the bounds with area 0.  A
    doubly wound square alone in an atlas it exactly fills at scale 1 is the
    case an uncertified bound would get wrong (twice its area exceeds the
    atlas); with a pentagram and a bow tie beside it, single packs and a
    batch with the progressive bound all give the oracle's scale and
    placements."""
    s = 100 * 256
    square = [(0, 0), (s, 0), (s, s), (0, s)]
    cs = synth.from_polygons([_looped(square, 2)], 100, 100)
    p = gpu_params()
    o = _compare_pack(cs, ctx.pack(cs, p), oracle_params(p))
    assert o.k == 1024
    pent = [(int(12800 + 12000 * np.sin(2 * np.pi * 2 * i / 5)), int(12800 - 12000 * np.cos(2 * np.pi * 2 * i / 5)))
            for i in range(5)]  # a pentagram: its centre is wound twice
    bow = [(0, 0), (s // 2, s // 2), (s // 2, 0), (0, s // 2)]
    mixed = synth.from_polygons([_looped(square, 3), pent, bow, _looped(pent, 2)], 160, 130)
    for fanout in (64, 8):
        p = gpu_params(scale_fanout=fanout)
        _compare_pack(mixed, ctx.pack(mixed, p), oracle_params(p))
    sets = [cs, mixed, synth.stars(31, 300, 512)]
    shape = tabi.Tuning(scale_fanout=2, raster_warp_items=32768, rowloop_threads=1024, rowloop_ctas=1,
                        chunks=4, progressive_bound=1)
    st, res = ctx.pack_batch(sets, gpu_params(), shape=shape)
    assert st == tabi.TABI_OK
    for c, r in zip(sets, res):
        _compare_pack(c, r, oracle_params(gpu_params()))


def test_invalid_inputs(ctx):
    p = gpu_params()
    bad = [synth.from_polygons([[(0, 0), (100, 0), (100, 600)]], 32, 32),      # < 1 texel wide
           synth.from_polygons([[(0, 0), (1 << 20, 0), (0, 600)]], 32, 32)]    # out of range
    for cs in bad:
        assert ctx.pack(cs, p).status == tabi.TABI_ERR_INVALID_ARG
    cs = synth.rectangles([(3, 5)], 32, 32)
    cs.atlas_w = 0
    assert ctx.pack(cs, p).status == tabi.TABI_ERR_INVALID_ARG
    # the context still works afterwards
    cs = synth.rectangles([(3, 5)], 32, 32)
    assert ctx.pack(cs, p).status == tabi.TABI_OK


def test_device_entry_point_matches_host(ctx):
    cs = synth.knees(3, 400, 1024)
    p = gpu_params()
    host = ctx.pack(cs, p)
    dev = torch.device("cuda:0")
    offs = torch.from_numpy(cs.offsets.view(np.int32).copy()).to(dev)
    verts = torch.from_numpy(cs.verts.copy()).to(dev)
    out = torch.zeros(tabi.PLACEMENT_DTYPE.itemsize * cs.n, dtype=torch.uint8, device=dev)
    st, k = ctx.pack_device(cs.n, cs.nv, cs.atlas_w, cs.atlas_h, offs, verts, out, p)
    torch.cuda.synchronize()
    assert st == 0 and k == host.k
    got = out.cpu().numpy().view(tabi.PLACEMENT_DTYPE)
    assert np.array_equal(got, host.place)


def test_deterministic(ctx):
    cs = synth.stars(12, 700, 1024)
    p = gpu_params()
    a = ctx.pack(cs, p)
    b = ctx.pack(cs, p)
    assert a.k == b.k and np.array_equal(a.place, b.place)


def test_small_arena_reports_oom():
    c = tabi.Context(arena_bytes=2 << 20)
    try:
        cs = synth.stars2k()
        assert c.pack(cs, gpu_params()).status == tabi.TABI_ERR_OOM
    finally:
        c.close()
