"""GPU parity of the batched form: many atlases of uneven size packed by one
launch sequence (tabi_pack_batch / tabi_pack_batch_device), each bit-exact
with the CPU oracle and identical to the same atlas packed alone.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # the -m gpu suite runs on a GPU machine only
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_2602_07782_gb300 import tabi  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = tabi.Context(arena_bytes=4 << 30)
    yield c
    c.close()


def oracle_params(p):
    return oracle.default_params(gutter=p.gutter, knee_abs=p.knee_abs_pct, knee_rel=p.knee_rel_pct,
                                 lr_sig=p.lr_sig_pct, knee_margin=p.knee_margin, flags=p.flags & tabi.F_ALL,
                                 laabb_k=p.laabb_count, topt=p.topt_permille, hybrid_min=p.hybrid_min_charts)


def mixed_batch():
    """Uneven chart counts and atlas sizes, knees, a non-square atlas."""
    sets = [synth.plain64(seed=1), synth.stars(3, 300, 512), synth.knees(1, 300, 1024),
            synth.knees(5, 200, 512), synth.pareto20k(seed=9, n=1500, atlas=1024),
            synth.stars(8, 40, 256), synth.rectangles([(7, 7)] * 50, 100, 60)]
    cs = synth.knees(7, 123, 777)
    cs.atlas_h = 333
    sets.append(cs)
    return sets


def compare(cs, res, op):
    o = oracle.pack(cs, op)
    assert res.status == {0: 0, 2: 2, 1: 1}[o.status], cs.name
    assert res.k == o.k, cs.name
    if o.status == 0:
        pl = res.place
        for f, col in (("x", 0), ("y", 1), ("rot90", 2), ("flip_x", 3), ("flip_y", 4), ("mirror", 5), ("k", 10)):
            assert np.array_equal(pl[f], o.place[:, col]), (cs.name, f)


@pytest.mark.parametrize("fanout", [64, 8, 5, 1])
def test_batch_parity(ctx, fanout):
    sets = mixed_batch()
    p = tabi.params_default(scale_fanout=fanout)
    st, res = ctx.pack_batch(sets, p)
    assert st == tabi.TABI_OK, ctx.last_error()
    op = oracle_params(p)
    for cs, r in zip(sets, res):
        compare(cs, r, op)


SHAPES = [  # (fan-out, raster warp-items, row-loop threads, CTAs per SM, chunks, progressive bound)
    (2, 32768, 1024, 1, 4, 1), (2, 65536, 1024, 1, 6, 1), (1, 16384, 1024, 1, 8, 1), (3, 32768, 512, 2, 2, 1),
    (8, 4096, 512, 1, 1, 0), (64, 32768, 1024, 1, 8, 0), (5, 100, 1024, 1, 3, 1), (16, 32768, 512, 2, 7, 0),
]


@pytest.mark.parametrize("shape", SHAPES, ids=[",".join(map(str, s)) for s in SHAPES])
def test_every_launch_shape_gives_the_oracle_result(ctx, shape):
    """No launch shape changes a result: each one, forced through
    tabi_pack_batch_shaped, packs every atlas of a batch exactly as the
    oracle does."""
    sets = mixed_batch()
    t = tabi.Tuning(*shape, 0.0)
    p = tabi.params_default()
    st, res = ctx.pack_batch(sets, p, shape=t)
    assert st == tabi.TABI_OK, ctx.last_error()
    op = oracle_params(p)
    for cs, r in zip(sets, res):
        compare(cs, r, op)


@pytest.mark.parametrize("shape", SHAPES[:4], ids=[",".join(map(str, s)) for s in SHAPES[:4]])
def test_batch_tail_in_chunks(ctx, shape):
    """The prefix-sum tail (Sec. 4.4) under lazy chunks: a task parks its
    tail state between chunks and resumes it; every atlas as the oracle
    packs it."""
    sets = mixed_batch()
    p = tabi.params_default(topt_permille=40, hybrid_min_charts=100)
    st, res = ctx.pack_batch(sets, p, shape=tabi.Tuning(*shape, 0.0))
    assert st == tabi.TABI_OK, ctx.last_error()
    op = oracle_params(p)
    for cs, r in zip(sets, res):
        compare(cs, r, op)


@pytest.mark.parametrize("count", [2, 5])
def test_batch_laabb_counts(ctx, count):
    """Tab. 13's local-AABB counts through the captured batch graph (the
    count picks its prep kernel): every atlas as the oracle packs it at that
    count, then at the default count again (a graph of its own)."""
    sets = mixed_batch()
    for c in (count, 10):
        p = tabi.params_default(laabb_count=c)
        st, res = ctx.pack_batch(sets, p)
        assert st == tabi.TABI_OK, ctx.last_error()
        op = oracle_params(p)
        for cs, r in zip(sets, res):
            compare(cs, r, op)


@pytest.mark.parametrize("gutter", [0, 2, 3])
def test_batch_gutters_with_the_progressive_bound(ctx, gutter):
    """The area bounds at other gutters (their g terms): a batch with the
    progressive bound on, every atlas as the oracle packs it."""
    sets = mixed_batch()
    p = tabi.params_default(gutter=gutter)
    st, res = ctx.pack_batch(sets, p, shape=tabi.Tuning(2, 32768, 1024, 1, 4, 1, 0.0))
    assert st == tabi.TABI_OK, ctx.last_error()
    op = oracle_params(p)
    for cs, r in zip(sets, res):
        compare(cs, r, op)


def test_bad_launch_shapes_are_refused(ctx):
    sets = mixed_batch()[:2]
    p = tabi.params_default()
    for bad in [(0, 32768, 1024, 1, 4, 1), (2, 0, 1024, 1, 4, 1), (2, 32768, 256, 1, 4, 1),
                (2, 32768, 1024, 3, 4, 1), (2, 32768, 1024, 1, 9, 1), (2, 32768, 1024, 1, 4, 2)]:
        st, _ = ctx.pack_batch(sets, p, shape=tabi.Tuning(*bad, 0.0))
        assert st == tabi.TABI_ERR_INVALID_ARG, bad


def test_batch_same_as_alone(ctx):
    sets = mixed_batch()
    p = tabi.params_default(scale_fanout=8)
    alone = [ctx.pack(cs, p) for cs in sets]
    st, res = ctx.pack_batch(sets[::-1], p)  # another order, too
    assert st == tabi.TABI_OK
    for a, b in zip(alone, res[::-1]):
        assert a.status == b.status and a.k == b.k
        assert np.array_equal(a.place, b.place)


def test_batch_steps_per_atlas(ctx):
    """Inspection of each atlas of a batch: prep, sort, envelopes, pairs and
    every candidate's row loop against the oracle."""
    sets = [synth.stars(3, 120, 512), synth.knees(5, 90, 512), synth.plain64(seed=2)]
    # one wave of all 64 candidates: no later wave reuses their regions
    p = tabi.params_default(flags=tabi.F_ALL | tabi.F_EVAL_ALL, scale_fanout=64)
    op = oracle_params(p)
    st, res = ctx.pack_batch(sets, p)
    assert st == tabi.TABI_OK
    for a, cs in enumerate(sets):
        rec = oracle.prep(cs, op)
        perm = ctx.perm(a)
        assert np.array_equal(perm, oracle.sort(rec))
        assert np.array_equal(ctx.charts(a)["Hq"].astype(np.int64), rec[:, oracle.R["HQ"]])
        for j in range(0, 64, 9):
            k = 16 * (j + 1)
            env = ctx.envelopes(j, cs.n, a)
            for s in range(cs.n):
                e = oracle.envelope_padded(rec[perm[s]], k, op)
                wp, hp, top, bot, left, right, mb = env[s]
                assert (wp, hp) == (e.w, e.h)
                assert np.array_equal(top, e.top) and np.array_equal(bot, e.bot)
                assert np.array_equal(left, e.left) and np.array_equal(right, e.right)
            d, ca, cb = ctx.pairs(j, cs.n, a)
            od, oca, ocb, _, _ = oracle.scale_pairs(rec, perm, k, op)
            assert np.array_equal(d[:-1], od[:-1]) and d[-1] == 0
            assert np.array_equal(ca[:-1], oca[:-1]) and np.array_equal(cb[:-1], ocb[:-1])
            hdr, place = ctx.scale_result(j, cs.n, a)
            ok, opl, ost = oracle.pack_scale(rec, perm, cs.atlas_w, cs.atlas_h, k, op)
            assert hdr[0] == int(ok) and list(hdr[1:6]) == [int(v) for v in ost[:5]]
            assert hdr[6] == 1  # ran to its end
            placed = int(ost[4])
            assert np.array_equal(place[:placed, 0], opl[:placed, 0])
            assert np.array_equal(place[:placed, 1], opl[:placed, 1])


def test_batch_regions_tile_the_pools(ctx):
    """Within a wave (ranks wF .. wF+F-1 below each atlas's top candidate)
    the (atlas, candidate) regions are disjoint, 16-byte aligned and sized
    by the atlas's charts."""
    sets = mixed_batch()
    F = 8
    p = tabi.params_default(scale_fanout=F)
    st, _ = ctx.pack_batch(sets, p)
    assert st == tabi.TABI_OK
    info = [ctx.regions(a) for a in range(len(sets))]
    for which in (0, 1):
        for w in range(0, 64 // F):
            iv = []
            for starts, words, jtop in info:
                for r in range(w * F, (w + 1) * F):
                    if jtop - r >= 0:
                        iv.append((int(starts[jtop - r, which]), int(words[jtop - r, which])))
            iv.sort()
            for (s0, n0), (s1, _) in zip(iv, iv[1:]):
                assert s0 + n0 <= s1
            assert all(s % 4 == 0 and n % 4 == 0 for s, n in iv)


@pytest.mark.parametrize("fanout", [2, 5])
def test_wave_loop_stops_when_no_atlas_searches(ctx, fanout):
    """The graph's device-side wave loop runs exactly the waves the slowest
    atlas needs (down to the wave holding its result, or through its last
    candidate when nothing fits); direct launches run every wave."""
    sets = mixed_batch()
    p = tabi.params_default(scale_fanout=fanout)
    st, res = ctx.pack_batch(sets, p)
    assert st == tabi.TABI_OK
    need = 0
    for a, r in enumerate(res):
        jt = ctx.regions(a)[2]
        if r.status == tabi.TABI_OK:
            need = max(need, (jt - (r.k // 16 - 1)) // fanout + 1)
        elif r.status == tabi.TABI_ERR_NO_FIT and jt >= 0:
            need = max(need, jt // fanout + 1)
    assert ctx.waves_run() == max(1, need)
    ctx.stage_times(True)
    try:
        st, res2 = ctx.pack_batch(sets, p)
    finally:
        ctx.stage_times(False)
    assert st == tabi.TABI_OK and [r.k for r in res2] == [r.k for r in res]
    assert ctx.waves_run() == (64 + fanout - 1) // fanout


def test_envelopes_exist_up_to_the_top_candidate_only(ctx):
    """Candidates above the area bound's top are never evaluated: their
    envelopes are refused by inspection, the top candidate's are not."""
    cs = synth.stars(3, 300, 512)
    st, _ = ctx.pack_batch([cs, synth.plain64(seed=1)], tabi.params_default())
    assert st == tabi.TABI_OK
    jt = ctx.regions(0)[2]
    assert 0 <= jt < 63
    ctx.envelopes(jt, cs.n, 0)
    with pytest.raises(RuntimeError):
        ctx.envelopes(jt + 1, cs.n, 0)


def test_area_bound_keeps_the_result(ctx):
    """The top candidate the area bound allows is at least the chosen scale,
    and every candidate above it fails in the oracle too."""
    sets = mixed_batch()[:5]
    p = tabi.params_default()
    st, res = ctx.pack_batch(sets, p)
    assert st == tabi.TABI_OK
    op = oracle_params(p)
    for a, (cs, r) in enumerate(zip(sets, res)):
        jtop = ctx.regions(a)[2]
        assert r.k <= 16 * (jtop + 1)
        if jtop < 63:
            rec = oracle.prep(cs, op)
            perm = oracle.sort(rec)
            ok, _, _ = oracle.pack_scale(rec, perm, cs.atlas_w, cs.atlas_h, 16 * (jtop + 2), op)
            assert not ok


def test_progressive_area_bound_stops_only_failing_candidates(ctx):
    """Every candidate up to the area bound's top in one wave: each one that
    ends without success -- some stopped by the progressive area bound
    before their rows overflow -- fails in the oracle too, and the bound
    does stop some of them early."""
    sets = mixed_batch()[:5] + [synth.stars(21, 600, 1024), synth.stars(22, 900, 1024)]
    p = tabi.params_default(scale_fanout=64)
    st, res = ctx.pack_batch(sets, p)
    assert st == tabi.TABI_OK
    op = oracle_params(p)
    early = 0
    for a, (cs, r) in enumerate(zip(sets, res)):
        compare(cs, r, op)
        jtop = ctx.regions(a)[2]
        rec = oracle.prep(cs, op)
        perm = oracle.sort(rec)
        for j in range(jtop, -1, -1):
            hdr, _ = ctx.scale_result(j, cs.n, a)
            if hdr[6] != 1 or hdr[0]:
                continue  # abandoned, or successful
            ok, _, ost = oracle.pack_scale(rec, perm, cs.atlas_w, cs.atlas_h, 16 * (j + 1), op)
            assert not ok, (cs.name, j)
            early += int(hdr[5] < int(ost[4]))  # stopped with fewer charts placed than at the overflow
    assert early > 0


def test_batch_rejects_bad_requests_alone(ctx):
    """A request that fails the host checks, and one with an invalid chart,
    fail alone; the other atlases of the batch are unaffected."""
    good = [synth.stars(3, 300, 512), synth.plain64(seed=1)]
    bad_host = synth.rectangles([(3, 5)], 32, 32)
    bad_host.atlas_w = 0
    bad_dev = synth.from_polygons([[(0, 0), (100, 0), (100, 600)]], 32, 32)
    sets = [good[0], bad_host, bad_dev, good[1]]
    p = tabi.params_default()
    st, res = ctx.pack_batch(sets, p)
    assert st == tabi.TABI_OK
    assert res[1].status == tabi.TABI_ERR_INVALID_ARG and res[2].status == tabi.TABI_ERR_INVALID_ARG
    op = oracle_params(p)
    compare(good[0], res[0], op)
    compare(good[1], res[3], op)


def test_batch_device_entry_point(ctx):
    sets = mixed_batch()[:5]
    p = tabi.params_default(scale_fanout=16)
    st, host = ctx.pack_batch(sets, p)
    assert st == tabi.TABI_OK
    dev = torch.device("cuda:0")
    keep, reqs = [], (tabi.Request * len(sets))()
    for i, cs in enumerate(sets):
        offs = torch.from_numpy(cs.offsets.view(np.int32).copy()).to(dev)
        verts = torch.from_numpy(cs.verts.copy()).to(dev)
        out = torch.zeros(tabi.PLACEMENT_DTYPE.itemsize * cs.n, dtype=torch.uint8, device=dev)
        keep.append((offs, verts, out))
        reqs[i] = tabi.Request(cs.atlas_w, cs.atlas_h, cs.n, cs.nv, offs.data_ptr(), verts.data_ptr(),
                               out.data_ptr(), 0, 0)
    assert ctx.pack_batch_requests(reqs, p, device=True) == tabi.TABI_OK
    torch.cuda.synchronize()
    for i, h in enumerate(host):
        assert reqs[i].status == h.status and reqs[i].scale_k == h.k
        got = keep[i][2].cpu().numpy().view(tabi.PLACEMENT_DTYPE)
        assert np.array_equal(got, h.place)


def _device_requests(sets):
    dev = torch.device("cuda:0")
    keep, reqs = [], (tabi.Request * len(sets))()
    for i, cs in enumerate(sets):
        offs = torch.from_numpy(cs.offsets.view(np.int32).copy()).to(dev)
        verts = torch.from_numpy(cs.verts.copy()).to(dev)
        out = torch.zeros(tabi.PLACEMENT_DTYPE.itemsize * cs.n, dtype=torch.uint8, device=dev)
        keep.append((offs, verts, out))
        reqs[i] = tabi.Request(cs.atlas_w, cs.atlas_h, cs.n, cs.nv, offs.data_ptr(), verts.data_ptr(),
                               out.data_ptr(), 0, 0)
    return keep, reqs


def test_autotune_keeps_results_exact(ctx):
    """After the autotuner's trial launches (fan-outs, raster warp-items,
    512-thread row-loop CTAs two per multiprocessor) the requests hold the
    chosen shape's results, identical to the oracle's; the tuned shape is
    then used for fan-out 0."""
    sets = mixed_batch()
    keep, reqs = _device_requests(sets)
    p = tabi.params_default()
    st, t = ctx.autotune(reqs, p)
    assert st == tabi.TABI_OK, ctx.last_error()
    assert t.scale_fanout in (64, 16, 8, 4) and t.raster_warp_items in (16384, 32768, 65536)
    assert (t.rowloop_threads, t.rowloop_ctas) in ((1024, 1), (512, 2), (512, 1))
    assert t.ms > 0
    torch.cuda.synchronize()
    op = oracle_params(p)
    for i, cs in enumerate(sets):
        place = keep[i][2].cpu().numpy().view(tabi.PLACEMENT_DTYPE)
        compare(cs, tabi.PackResult(reqs[i].status, reqs[i].scale_k, place), op)
    # fan-out 0 takes the tuned shape; same results again
    st2, res = ctx.pack_batch(sets, p)
    assert st2 == tabi.TABI_OK
    for i, r in enumerate(res):
        assert r.status == reqs[i].status and r.k == reqs[i].scale_k


def test_batch_small_arena_fails_per_atlas():
    """Arenas too small for every region: the atlases whose regions do not
    fit report TABI_ERR_OOM, the others are still exact."""
    sets = [synth.stars(3, 300, 512), synth.stars2k(), synth.plain64(seed=1)]
    need = sum(tabi.arena_bytes(cs) for cs in sets)
    p = tabi.params_default(scale_fanout=64)
    op = oracle_params(p)
    saw_oom = False
    for div in (4, 8, 16, 32, 64):
        c = tabi.Context(arena_bytes=max(need // div, 2 << 20))
        try:
            st, res = c.pack_batch(sets, p)
            if st == tabi.TABI_ERR_OOM:
                break  # the per-chart arrays alone no longer fit
            assert st == tabi.TABI_OK
            for cs, r in zip(sets, res):
                assert r.status in (tabi.TABI_OK, tabi.TABI_ERR_OOM)
                if r.status == tabi.TABI_OK:
                    compare(cs, r, op)
                else:
                    saw_oom = True
        finally:
            c.close()
    assert saw_oom


@pytest.mark.slow
def test_batch_uneven_sizes_full_shapes(ctx):
    """Sixteen atlases drawn like the 256-atlas batch workload (chart counts
    50-5,000, atlas sides 1024/2048/4096, star charts), in the launch
    configuration the benchmark times."""
    sets = synth.batch256(count=16)
    p = tabi.params_default(scale_fanout=8)
    st, res = ctx.pack_batch(sets, p)
    assert st == tabi.TABI_OK
    op = oracle_params(p)
    for cs, r in zip(sets, res):
        assert r.status == tabi.TABI_OK
        compare(cs, r, op)


def test_pinned_host_buffers_match(ctx):
    """tabi_pack_batch with pinned host buffers (the device reads and writes
    them directly) and with pageable ones (copy calls), mixed in one batch,
    and the same batch from device buffers: identical results.  The pinned
    arrays start at offsets 0, 4 and 8 bytes into their allocations, so the
    copy kernel meets unaligned starts too."""
    sets = mixed_batch()
    p = tabi.params_default()
    st, ref = ctx.pack_batch(sets, p)
    assert st == tabi.TABI_OK, ctx.last_error()
    hold = []
    reqs = (tabi.Request * len(sets))()
    outs = []
    for i, cs in enumerate(sets):
        pinned = i % 3 != 2  # every third request stays pageable
        sh = 4 * (i % 3)  # byte offset of the arrays in their allocations
        if pinned:
            ob = torch.zeros(4 * (cs.n + 1) + 16, dtype=torch.uint8).pin_memory()
            vb = torch.zeros(8 * cs.nv + 16, dtype=torch.uint8).pin_memory()
            out_b = torch.zeros(tabi.PLACEMENT_DTYPE.itemsize * cs.n + 16, dtype=torch.uint8).pin_memory()
            ob.numpy()[sh:sh + 4 * (cs.n + 1)] = cs.offsets.view(np.uint8)
            vb.numpy()[sh:sh + 8 * cs.nv] = cs.verts.view(np.uint8)
            hold.append((ob, vb, out_b))
            optr, vptr, outp = ob.data_ptr() + sh, vb.data_ptr() + sh, out_b.data_ptr() + sh
            outs.append(out_b.numpy()[sh:sh + tabi.PLACEMENT_DTYPE.itemsize * cs.n])
        else:
            o, v = np.ascontiguousarray(cs.offsets, np.uint32), np.ascontiguousarray(cs.verts, np.int32)
            out_np = np.zeros(tabi.PLACEMENT_DTYPE.itemsize * cs.n, np.uint8)
            hold.append((o, v, out_np))
            optr, vptr, outp = o.ctypes.data, v.ctypes.data, out_np.ctypes.data
            outs.append(out_np)
        reqs[i] = tabi.Request(cs.atlas_w, cs.atlas_h, cs.n, cs.nv, optr, vptr, outp, 0, 0)
    for _ in range(2):  # twice: the second batch reuses the context's arena
        assert ctx.pack_batch_requests(reqs, p, device=False) == tabi.TABI_OK, ctx.last_error()
        for i, (cs, r) in enumerate(zip(sets, ref)):
            assert reqs[i].status == r.status and reqs[i].scale_k == r.k, cs.name
            got = outs[i].view(tabi.PLACEMENT_DTYPE)
            for f in ("x", "y", "rot90", "flip_x", "flip_y", "mirror"):
                assert np.array_equal(got[f], r.place[f]), (cs.name, f)
        for o in outs:
            o[:] = 0


@pytest.mark.slow
def test_full_batch_in_the_benchmark_shape_sampled():
    """The whole 256-atlas workload (614,480 charts) in the launch shape the
    benchmark's autotuner picks (fan-out 2, 64K raster warp-items, 1024-thread
    row-loop CTAs, four chunks, progressive area bound): every atlas's scale
    and placements against the oracle for a sample of 32 atlases spread over
    the batch (largest, smallest and evenly spaced by chart count)."""
    sets = synth.stars_many(synth.batch256_specs())
    need = sum(tabi.arena_bytes(cs) for cs in sets)
    c = tabi.Context(arena_bytes=min(need, 32 << 30) + (64 << 20))
    try:
        p = tabi.params_default()
        st, res = c.pack_batch(sets, p, shape=tabi.Tuning(2, 65536, 1024, 1, 4, 1, 0.0))
        assert st == tabi.TABI_OK, c.last_error()
    finally:
        c.close()
    assert all(r.status == tabi.TABI_OK for r in res)
    by_n = sorted(range(len(sets)), key=lambda i: sets[i].n)
    pick = sorted({by_n[0], by_n[-1], *by_n[::8]})
    out = oracle.pack_many([sets[i] for i in pick], oracle_params(p))
    for i, (ost, ok, opl) in zip(pick, out):
        assert ost == 0 and res[i].k == ok, i
        pl = res[i].place
        for f, col in (("x", 0), ("y", 1), ("rot90", 2), ("flip_x", 3), ("flip_y", 4), ("mirror", 5)):
            assert np.array_equal(pl[f], opl[:, col]), (i, f)
