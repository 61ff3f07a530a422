"""GPU tests of the serving loop (tabi_server_*): requests submitted while
others are on the GPU are batched and overlapped, and every request gets
exactly the result it gets alone (and the oracle's, for the small ones).
"""
from __future__ import annotations

import random
import threading
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # the -m gpu suite runs on a GPU machine only
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_2602_07782_gb300 import tabi  # noqa: E402


def mix():
    sets = [synth.plain64(seed=s) for s in (1, 2, 3)]
    sets += [synth.stars(10 + i, n, side) for i, (n, side) in
             enumerate([(40, 256), (300, 512), (900, 1024), (1500, 1024), (2000, 2048), (120, 512)])]
    sets += [synth.knees(4, 250, 1024)]
    return sets


@pytest.fixture(scope="module")
def alone():
    c = tabi.Context(arena_bytes=2 << 30)
    p = tabi.params_default(scale_fanout=8)
    res = [c.pack(cs, p) for cs in mix()]
    c.close()
    return res


def test_served_results_equal_alone(alone):
    """A stream with random gaps and repeats: every completed request equals
    the same request packed alone; several batches and lanes were used."""
    sets = mix()
    srv = tabi.Server(lanes=3, max_batch=8, arena_bytes=3 << 30)
    try:
        rng = random.Random(7)
        order = [rng.randrange(len(sets)) for _ in range(60)]
        tickets = []

        def producer():
            # a burst (queued behind busy lanes: batched), then random gaps
            for n, i in enumerate(order):
                st, t, out = srv.submit(sets[i])
                assert st == tabi.TABI_OK
                tickets.append((i, t, out))
                if n >= 30:
                    time.sleep(rng.choice([0.0, 0.0, 0.0005, 0.002]))

        th = threading.Thread(target=producer)
        th.start()
        th.join()
        for i, t, out in tickets:
            st, r = srv.wait(t, 60000)
            assert st == tabi.TABI_OK
            assert r.status == alone[i].status and r.scale_k == alone[i].k
            assert np.array_equal(out, alone[i].place)
            assert r.t_submit_ns <= r.t_start_ns <= r.t_done_ns
        stats = srv.stats()
        assert stats["completed"] == len(order) and stats["queued"] == 0
        assert stats["batches"] >= 2 and stats["max_batch"] >= 2
    finally:
        srv.close()


def test_served_small_requests_match_oracle():
    sets = [synth.plain64(seed=s) for s in (4, 5)] + [synth.stars(31, 150, 512)]
    srv = tabi.Server(lanes=2, max_batch=4, arena_bytes=1 << 30)
    try:
        subs = [srv.submit(cs) for cs in sets]
        for cs, (st, t, out) in zip(sets, subs):
            st, r = srv.wait(t)
            assert st == tabi.TABI_OK and r.status == tabi.TABI_OK
            o = oracle.pack(cs)
            assert r.scale_k == o.k
            assert np.array_equal(out["x"], o.place[:, 0]) and np.array_equal(out["y"], o.place[:, 1])
            assert np.array_equal(out["mirror"], o.place[:, 5])
    finally:
        srv.close()


def test_served_bad_and_oversized_requests_fail_alone(alone):
    sets = mix()
    srv = tabi.Server(lanes=2, max_batch=16, arena_bytes=64 << 20)
    try:
        bad = synth.from_polygons([[(0, 0), (100, 0), (100, 600)]], 32, 32)  # < 1 texel wide
        big = synth.stars(77, 2000, 2048)                                     # more than a lane holds
        st_b, t_b, _ = srv.submit(bad)
        st_g, t_g, _ = srv.submit(big)
        st_s, t_s, out_s = srv.submit(sets[0])
        assert st_b == st_g == st_s == tabi.TABI_OK
        assert srv.wait(t_b)[1].status == tabi.TABI_ERR_INVALID_ARG
        assert srv.wait(t_g)[1].status == tabi.TABI_ERR_OOM
        st, r = srv.wait(t_s)
        assert r.status == alone[0].status and r.scale_k == alone[0].k
        assert np.array_equal(out_s, alone[0].place)
    finally:
        srv.close()


def test_submit_checks_offsets_before_reading_vertices():
    """The server walks a request's vertex loops on the host to size it, so
    tabi_submit checks the offsets first: a middle offset past n_verts, a
    decreasing one, or a chart with fewer than three vertices completes the
    ticket with TABI_ERR_INVALID_ARG instead of reading out of bounds."""
    srv = tabi.Server(lanes=1, max_batch=4, arena_bytes=256 << 20)
    try:
        verts = np.array([0, 0, 512, 0, 512, 512, 0, 0, 512, 0, 512, 512], np.int32)
        for offs in ([0, 1 << 30, 6], [0, 4, 2, 6], [0, 2, 6], [0, 6, 6]):
            o = np.array(offs, np.uint32)
            out = np.zeros(len(offs) - 1, tabi.PLACEMENT_DTYPE)
            st, t, _ = srv.submit_ptrs(len(offs) - 1, 6, 64, 64, o, verts, out)
            assert st == tabi.TABI_OK
            st, r = srv.wait(t)
            assert st == tabi.TABI_OK and r.status == tabi.TABI_ERR_INVALID_ARG, offs
        good = np.array([0, 3, 6], np.uint32)
        st, t, out = srv.submit_ptrs(2, 6, 64, 64, good, verts, np.zeros(2, tabi.PLACEMENT_DTYPE))
        assert srv.wait(t)[1].status == tabi.TABI_OK
    finally:
        srv.close()


def test_poll_wait_and_unknown_tickets():
    srv = tabi.Server(lanes=1, max_batch=4, arena_bytes=512 << 20)
    try:
        st, t, _ = srv.submit(synth.stars(5, 800, 1024))
        assert st == tabi.TABI_OK
        st, _ = srv.poll(t)
        assert st in (tabi.TABI_PENDING, tabi.TABI_OK)
        if st == tabi.TABI_PENDING:
            st, r = srv.wait(t, 60000)
            assert st == tabi.TABI_OK and r.status == tabi.TABI_OK
        assert srv.poll(t)[0] == tabi.TABI_ERR_INVALID_ARG  # released
        assert srv.poll(123456789)[0] == tabi.TABI_ERR_INVALID_ARG
    finally:
        srv.close()


def test_shutdown_with_requests_queued_is_bounded():
    """Closing a server with requests queued and in flight returns; nothing
    waits on the device without a bound."""
    srv = tabi.Server(lanes=1, max_batch=1, arena_bytes=512 << 20)
    cs = synth.stars(6, 600, 1024)
    for _ in range(20):
        assert srv.submit(cs)[0] == tabi.TABI_OK
    t0 = time.time()
    srv.close()
    assert time.time() - t0 < 60


def test_served_stream_sample_matches_oracle():
    """A sample of the benchmark's served stream -- its own request bodies
    (stars_fast over serve_specs), every atlas side, chart counts up to the
    prefix-sum tail's range -- through the server in the benchmark's
    configuration (4 lanes over 8 GiB, fan-out 8, the overlap counter on),
    all submitted at once so they share batches: each result is the
    oracle's, and its overlap, gutter and outside counts are zero."""
    specs = synth.serve_specs()
    picked, seen = [], set()
    for t, seed, n, side in specs:
        cls = (side, n > 10000, n > 2000)
        if cls not in seen and n <= 14000:
            seen.add(cls)
            picked.append(synth.stars_fast(seed, n, side))
    assert any(cs.n > 10000 for cs in picked) and len({cs.atlas_w for cs in picked}) == 4
    srv = tabi.Server(lanes=4, max_batch=64, arena_bytes=8 << 30,
                      params=tabi.params_default(scale_fanout=8), check=1)
    try:
        subs = [srv.submit(cs) for cs in picked]
        got = []
        for st, t, out in subs:
            assert st == tabi.TABI_OK
            st, r = srv.wait(t, 120000)
            assert st == tabi.TABI_OK and r.status == tabi.TABI_OK
            assert (r.overlap_texels, r.gutter_texels, r.outside_texels) == (0, 0, 0)
            got.append((r.scale_k, out.copy()))
    finally:
        srv.close()
    ref = oracle.pack_many(picked)
    for cs, (k, out), (st, ko, place) in zip(picked, got, ref):
        assert st == 0 and k == ko, cs.name
        assert np.array_equal(out["x"], place[:, 0]) and np.array_equal(out["y"], place[:, 1]), cs.name
        assert np.array_equal(out["mirror"], place[:, 5]) and np.array_equal(out["k"], place[:, 10]), cs.name
