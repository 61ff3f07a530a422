"""Benchmark of the GB300 atlas packer: the batched form.

Workload: 256 independent atlases (chart counts uniform in 50..5,000, atlas
sides drawn from 1024/2048/4096, star-shaped charts with 6-64 vertices,
log-normal areas sigma 1.0, aspect 1:1-1:8), packed together by one launch
sequence replayed from a captured CUDA graph, 1-px gutters, 64 candidate
scales per atlas.  One step = one such batch: every stage of the hot path
(prep, sort, envelope raster, compaction, row loop, selection) for all 256
atlases.  The launch shape is autotuned once before timing (tabi_autotune;
no knob changes a result).

Prints one JSON line.  value: atlases packed per second, inputs resident in
HBM, L2 flushed (256 MiB write) before every step, each step bracketed by
CUDA events on the packing stream.  e2e: the same batch through the
host-buffer entry point (tabi_pack_batch) from pinned host memory, the
host<->device copies inside the timed region.  plain: the same atlases
through the single-atlas entry point, one call each.  served: the serving
loop (tabi_server, continuous batching, 8 GiB arena) under a Poisson
stream of 2,000 requests/s for 10 s (chart counts log-uniform 16..20,000,
sides 512..4096), p50/p99 latency against the 15 ms interactive budget,
beside the plain packer serving the same stream one request at a time.  The roofline stage
times come from CUDA events the library records on the packing stream
around every stage, over K further steps of the same workload.
--impl reference times the CPU oracle on the same atlases.

Multi-GPU: atlases are independent, so every rank packs its own copy of the
batch (weak scaling, no collective on the data path); value = atlases of
all ranks / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = ("batch256: 256 atlases, chart counts U[50,5000], sides {1024,2048,4096}^2, star charts "
            "(6-64 verts, lognormal areas s=1.0, aspect 1:1-1:8), one batched pack per step")
METRIC = "packs/sec and p50/p99 ms per atlas, batched/served vs plain GPU packer"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--atlases", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--fanout", type=int, default=0,
                    help="with --no-autotune: candidates per wave (0: the library default)")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-bodies", type=int, default=256)
    ap.add_argument("--serve-lanes", type=int, default=4)
    ap.add_argument("--serve-fanout", type=int, default=8)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.rows.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 3 + i and "Active" in r[3 + i]
                          and "Not" not in r[3 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def workload(count: int):
    import synth
    return synth.stars_many(synth.batch256_specs(count=count))


def cpu_baseline(sets, budget_s: float = 15.0):
    """The oracle as it stands (single-threaded C, descending candidates until
    the first success), on the batch's atlases in order until the budget."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    packs = charts = 0
    for cs in sets:
        r = oracle.pack(cs)
        assert r.status == 0
        packs += 1
        charts += cs.n
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": packs / dt, "unit": "packs/s", "cores": 1, "kind": "oracle",
            "sample": f"the first {packs} atlases of the batch ({charts} charts), {dt:.1f} s on one host core"}


# DRAM read + write of every raster_kernel launch of one batch of this
# workload (ncu, direct launches, the launch shape below), with a digest of
# the kernel's sources at capture time; the bench reports it per launch
# while the sources and the shape match, else null.
RASTER_NCU = {"dram_bytes_per_step": 2676225280, "sources_sha256_16": "769f1f70cd681781",
              "shape": {"scale_fanout": 2, "chunks": 4, "progressive_bound": 1}}


def raster_sources_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("raster.cu", "raster_math.cuh"):
        with open(os.path.join(ROOT, "paper_2602_07782_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


SMS = 152  # multiprocessors of a GB300


def raster_ops_per_word(g: int) -> int:
    """Integer operations one padded scanline word of an envelope needs by
    its definition (App. A proxies, Sec. 5 gutter): ten local-AABB pieces,
    each a subtract, an unsigned range compare, a min and a max (40); two
    OBB bounds, each the extreme of two lines (a multiply-add and an exact
    division by multiply-high, shift and subtract per line, then a max or
    min: 9) and the corner override (two compares and a select: 3) (24);
    the combination with the pieces and the clamps to the chart box (6);
    the gutter dilation, a min and a max per neighbour over 2g neighbours
    (4g); packing the word and the deepest bottom (3)."""
    return 40 + 24 + 6 + 4 * g + 3


def max_over_ranks(total_ms: float, world: int, device=None) -> float:
    """The timed region of the slowest replica (whole-job time): a MAX
    all-reduce over the ranks (NCCL on the GPUs, gloo in the CPU tests)."""
    if world <= 1:
        return total_ms
    import torch
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def wave_ranges(jtop: int, k_best: int, F: int):
    """(wave, candidates) the batch evaluates for one atlas: waves of F
    candidates below its top candidate, down to the wave of its result."""
    j_best = k_best // 16 - 1 if k_best > 0 else -1
    out = []
    w = 0
    while jtop - w * F >= 0:
        hi = jtop - w * F
        lo = max(0, hi - F + 1)
        out.append((w, list(range(lo, hi + 1))))
        if lo <= j_best:
            break
        w += 1
    return out


def algorithmic_bytes(sets, ks, jtops, F, g=1):
    """Unavoidable HBM bytes of the raster and compaction stages of one batch
    (per chart and evaluated candidate: the envelope words it writes, its
    per-candidate offsets and meta; per chart and wave: its 208-byte shape
    record), from the charts' AABBs."""
    raster = hcomp = 0
    for cs, k_best, jt in zip(sets, ks, jtops):
        v = cs.verts.reshape(-1, 2).astype(np.int64)
        seg = np.repeat(np.arange(cs.n), np.diff(cs.offsets.astype(np.int64)))
        mn = np.full((cs.n, 2), np.iinfo(np.int64).max)
        mx = np.full((cs.n, 2), np.iinfo(np.int64).min)
        np.minimum.at(mn, seg, v)
        np.maximum.at(mx, seg, v)
        ext = mx - mn
        wq = np.minimum(ext[:, 0], ext[:, 1])
        hq = np.maximum(ext[:, 0], ext[:, 1])
        for _, js in wave_ranges(jt, k_best, F):
            raster += 208 * cs.n
            for j in js:
                k = 16 * (j + 1)
                wp = ((wq * k + (1 << 18) - 1) >> 18) + 2 * g
                hp = ((hq * k + (1 << 18) - 1) >> 18) + 2 * g
                # columns + their owners, rows, meta, column / row offsets
                raster += int(8 * wp.sum() + 4 * hp.sum()) + (16 + 8) * cs.n
                # rows read once, meta read, distance and flags written
                hcomp += int(4 * hp.sum()) + (16 + 4 + 4 + 1) * cs.n
    return {"raster": raster, "hcompact": hcomp}


def device_requests(tabi, torch, dev, sets):
    keep, reqs = [], (tabi.Request * len(sets))()
    for i, cs in enumerate(sets):
        offs = torch.from_numpy(cs.offsets.view(np.int32).copy()).to(dev)
        verts = torch.from_numpy(cs.verts.copy()).to(dev)
        out = torch.zeros(tabi.PLACEMENT_DTYPE.itemsize * cs.n, dtype=torch.uint8, device=dev)
        keep.append((offs, verts, out))
        reqs[i] = tabi.Request(cs.atlas_w, cs.atlas_h, cs.n, cs.nv, offs.data_ptr(), verts.data_ptr(),
                               out.data_ptr(), 0, 0)
    return keep, reqs


def run_ours(args, rank, world, local, sets):
    import torch

    from paper_2602_07782_gb300 import tabi

    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    A = len(sets)
    need = sum(tabi.arena_bytes(cs) for cs in sets)
    ctx = tabi.Context(arena_bytes=min(need, 32 << 30), device=local)
    stream = torch.cuda.Stream(device=dev)
    keep, reqs = device_requests(tabi, torch, dev, sets)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    params = tabi.params_default()  # fan-out 0: the tuned launch shape
    if not args.no_autotune:
        st, t = ctx.autotune(reqs, params, stream=stream)
        assert st == 0, ctx.last_error()
        tuning = {"scale_fanout": t.scale_fanout, "raster_warp_items": t.raster_warp_items,
                  "rowloop_threads": t.rowloop_threads, "rowloop_ctas": t.rowloop_ctas,
                  "chunks": t.chunks, "progressive_bound": t.progressive_bound,
                  "tuned_batch_ms": round(t.ms, 3)}
    else:  # the library's default shape for a batch, or the given fan-out
        params.scale_fanout = args.fanout
        tuning = {"scale_fanout": args.fanout or 8, "raster_warp_items": 32768, "rowloop_threads": 1024,
                  "rowloop_ctas": 1, "chunks": 4, "progressive_bound": 1, "autotuned": False}
    F, Q = tuning["scale_fanout"], tuning["chunks"]

    def step(ev=None):
        with torch.cuda.stream(stream):
            # evict L2 (129 MB) before the step, on the packing stream so the
            # write is ordered before the step's start event and kernels
            flush.fill_(1)
            if ev:
                ev[0].record(stream)
            st = ctx.pack_batch_requests(reqs, params, stream=stream)
            if ev:
                ev[1].record(stream)
        assert st == 0, ctx.last_error()

    for _ in range(args.warmup):
        step()
    ks = [r.scale_k for r in reqs]
    assert all(r.status == 0 for r in reqs)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    gpu_id = local
    if "CUDA_VISIBLE_DEVICES" in os.environ:
        try:
            gpu_id = int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local])
        except ValueError:
            pass

    # timed region: K batches (graph replay), events on the packing stream
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    with ClockSampler(gpu_id) as clk:
        t_wall = time.perf_counter()
        for i in range(args.steps):
            step(evs[i])
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    per = np.array([a.elapsed_time(b) for a, b in evs])
    waves_run = ctx.waves_run()  # waves of the graph's device-side loop in the last timed batch
    total_ms = float(per.sum())
    if world > 1:
        total_ms = max_over_ranks(total_ms, world, dev)
        torch.distributed.barrier()
    assert [r.scale_k for r in reqs] == ks

    # per-stage device time: library events around every stage, K steps
    ctx.stage_times(True)
    for i in range(args.steps):
        step()
    torch.cuda.synchronize()
    stage_ms, stage_launches, npacks = ctx.stage_times(False)

    # plain GPU packer on the same atlases: one tabi_pack_device call each
    plain_ms = []
    for i, cs in enumerate(sets):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, k = ctx.pack_device(cs.n, cs.nv, cs.atlas_w, cs.atlas_h, keep[i][0], keep[i][1], keep[i][2],
                                params, stream=stream)
        plain_ms.append(1e3 * (time.perf_counter() - t0))
        assert st == 0 and k == ks[i]
    plain_ms = np.array(plain_ms)

    # end to end through tabi_pack_batch: pinned host buffers, copies inside
    hold = []
    hreqs = (tabi.Request * A)()
    for i, cs in enumerate(sets):
        offs_h = torch.from_numpy(cs.offsets.view(np.int32).copy()).pin_memory()
        verts_h = torch.from_numpy(cs.verts.copy()).pin_memory()
        out_h = torch.zeros(tabi.PLACEMENT_DTYPE.itemsize * cs.n, dtype=torch.uint8).pin_memory()
        hold.append((offs_h, verts_h, out_h))
        hreqs[i] = tabi.Request(cs.atlas_w, cs.atlas_h, cs.n, cs.nv, offs_h.data_ptr(), verts_h.data_ptr(),
                                out_h.data_ptr(), 0, 0)
    e2e = []
    for i in range(args.warmup + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = ctx.pack_batch_requests(hreqs, params, stream=stream, device=False)
        dt = time.perf_counter() - t0
        assert st == 0 and [r.scale_k for r in hreqs] == ks
        if i >= args.warmup:
            e2e.append(dt)
    e2e_s = float(np.sum(e2e))
    h2d = int(sum(4 * (cs.n + 1) + 8 * cs.nv for cs in sets))
    d2h = int(sum(tabi.PLACEMENT_DTYPE.itemsize * cs.n for cs in sets)) + 16 * A

    # roofline of the dominant stage
    jtops = [ctx.regions(a)[2] for a in range(A)]
    alg = algorithmic_bytes(sets, ks, jtops, F)
    raster_words = ctx.raster_words()  # padded scanline words the (last, stage-timed) batch rasterized
    raster_cols = ctx.raster_column_words()
    # the raster's bytes from the words it evaluated: 8 B per column word
    # (word + owner index), 4 B per row word
    alg["raster"] = 8 * raster_cols + 4 * (raster_words - raster_cols)
    kernels = {s: stage_ms[s] for s in ("prep", "sort", "layout", "raster", "hcompact", "rowloop", "select")}
    dom = max(kernels, key=kernels.get)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    launches_dom = max(1, stage_launches[dom] // max(1, npacks))
    dom_ms = stage_ms[dom] / max(1, stage_launches[dom])
    dom_bytes = alg.get(dom, 0) / launches_dom
    achieved_gbs = dom_bytes / (dom_ms * 1e-3) / 1e9 if dom_ms > 0 and dom in alg else 0.0
    # traffic per launch: the captured launch's DRAM / algorithmic ratio
    # times this launch's algorithmic bytes, while the kernel is unchanged
    traffic = None
    if (dom == "raster" and RASTER_NCU and raster_sources_digest() == RASTER_NCU["sources_sha256_16"]
            and all(tuning.get(k) == v for k, v in RASTER_NCU["shape"].items())):
        traffic = int(RASTER_NCU["dram_bytes_per_step"] / launches_dom)
    hbm_view = {"kernel": dom, "bound": "hbm", "achieved": round(achieved_gbs, 2), "peak": hbm_peak,
                "unit": "GB/s", "frac": round(achieved_gbs / hbm_peak, 5), "traffic": traffic,
                "traffic_source": ("ncu capture of this workload's raster launches (profiles/raster_kernel_batch256.md)"
                                   if traffic else "null: no ncu capture of the current kernel at this launch shape"),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": int(dom_bytes), "avg_launch_ms": round(dom_ms, 4),
                "launches_per_step": int(launches_dom)}
    roofline = hbm_view
    if dom == "raster":
        # the raster is bound by integer issue (ncu: ALU pipe and issue slots
        # busiest, DRAM far from peak): algorithmic integer operations per
        # launch over its average event-timed launch, against the issue
        # rate of the multiprocessors at their maximum clock
        sm_max = (clk.summary().get("sm_max_mhz") or 2070.0)
        alu_peak = SMS * 4 * 32 * sm_max * 1e6 / 1e12  # tera lane-operations per second
        ops_launch = raster_words * raster_ops_per_word(1) / launches_dom
        achieved_t = ops_launch / (dom_ms * 1e-3) / 1e12 if dom_ms > 0 else 0.0
        roofline = {"kernel": "raster", "bound": "alu", "achieved": round(achieved_t, 4), "peak": round(alu_peak, 3),
                    "unit": "Tops/s", "frac": round(achieved_t / alu_peak, 5), "traffic": traffic,
                    "traffic_source": hbm_view["traffic_source"],
                    "peak_source": f"{SMS} SMs x 4 schedulers x 32 lanes x {sm_max:.0f} MHz (maximum SM clock)",
                    "ops_per_word": raster_ops_per_word(1), "words_per_step": int(raster_words),
                    "algorithmic_ops_per_launch": int(ops_launch), "avg_launch_ms": round(dom_ms, 4),
                    "launches_per_step": int(launches_dom), "hbm_view": hbm_view}

    res = {
        "metric": METRIC,
        "value": world * A * args.steps / (total_ms * 1e-3),
        "unit": "packs/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "p50_ms": float(np.percentile(per, 50)),
        "p99_ms": float(np.percentile(per, 99)),
        "latency_note": "batched: every atlas of a step completes with the step, so its latency is the step time",
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32/int64 (integer path)",
        "data": "synthetic (seeded star charts; the paper's chart sets are not available)",
        "config": {"workload": WORKLOAD, "atlases": A, "charts": int(sum(cs.n for cs in sets)),
                   "vertices": int(sum(cs.nv for cs in sets)), "candidates": 64, "gutter": 1,
                   "tuning": tuning, "waves_per_step": waves_run, "k_mean": float(np.mean(ks)),
                   "l2": "flushed before every step (256 MiB write), outside the timed events",
                   "parallelism": f"replicas x{world}"},
        "plain": {"value": A / (plain_ms.sum() * 1e-3), "unit": "packs/s",
                  "p50_ms": float(np.percentile(plain_ms, 50)), "p99_ms": float(np.percentile(plain_ms, 99)),
                  "how": "the same atlases, one tabi_pack_device call each (stream-synchronous), wall clock"},
        "e2e": {"value": world * A * args.steps / e2e_s, "unit": "packs/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(args.steps * tabi.kernels_per_pack(F, Q, waves_run)),
        "stages_ms_per_step": {s: round(stage_ms[s] / max(1, npacks), 4) for s in stage_ms},
        "roofline": roofline,
        "clocks": clk.summary(),
        "wall_s_timed_region": t_wall,
    }
    ctx.close()
    return res


def serve_workload(args):
    """Arrival times and request bodies of the served workload: Poisson
    arrivals at --serve-rate for --serve-seconds, chart counts log-uniform
    in 16..20,000, sides 512..4096, star charts; the arrivals draw their
    bodies from the first --serve-bodies distinct requests of the stream
    (generating all 20,000 bodies would take an hour of host time)."""
    import synth
    specs = synth.serve_specs(rate=args.serve_rate, duration=args.serve_seconds)
    P = min(args.serve_bodies, len(specs))
    bodies = synth.stars_many([sp[1:] for sp in specs[:P]])
    return [sp[0] for sp in specs], [i % P for i in range(len(specs))], bodies


def run_served(args, local, arrivals, body_of, bodies):
    """The serving loop under the Poisson stream: submit each request at its
    arrival time from one host thread, collect completions on another.
    Latency = result handed over - submitted (library host clock)."""
    import ctypes

    import torch

    from paper_2602_07782_gb300 import tabi
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    # each body alone through the plain single-atlas packer: its result and
    # its service time (stream-synchronous call, wall clock, median of 3)
    ctx = tabi.Context(arena_bytes=8 << 30, device=local)
    params = tabi.params_default()
    ref_k, service = [], []
    for cs in bodies:
        offs = torch.from_numpy(cs.offsets.view(np.int32).copy()).to(dev)
        verts = torch.from_numpy(cs.verts.copy()).to(dev)
        out = torch.zeros(tabi.PLACEMENT_DTYPE.itemsize * cs.n, dtype=torch.uint8, device=dev)
        ts = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, k = ctx.pack_device(cs.n, cs.nv, cs.atlas_w, cs.atlas_h, offs, verts, out, params)
            ts.append(time.perf_counter() - t0)
            assert st == 0, ctx.last_error()
        ref_k.append(k)
        service.append(float(np.median(ts)))
    ctx.close()
    # the plain packer serving the same stream: one pack at a time, FIFO
    done = 0.0
    plain_lat = []
    for t, b in zip(arrivals, body_of):
        done = max(done, t) + service[b]
        plain_lat.append(done - t)
    plain_lat = np.array(plain_lat) * 1e3
    plain_span = done - arrivals[0]

    sp = tabi.params_default(scale_fanout=args.serve_fanout)
    srv = tabi.Server(lanes=args.serve_lanes, max_batch=64, arena_bytes=8 << 30, params=sp)
    host = [(np.ascontiguousarray(cs.offsets, np.uint32), np.ascontiguousarray(cs.verts, np.int32)) for cs in bodies]
    for b, cs in enumerate(bodies):  # warm-up: every body once (graphs, caches)
        st, t, _ = srv.submit_ptrs(cs.n, cs.nv, cs.atlas_w, cs.atlas_h, host[b][0], host[b][1],
                                   np.zeros(cs.n, tabi.PLACEMENT_DTYPE))
        assert st == 0
    while srv.stats()["completed"] < len(bodies):
        time.sleep(0.01)
    base = srv.stats()
    tickets = [None] * len(arrivals)
    results = [None] * len(arrivals)
    ready = threading.Semaphore(0)

    def submitter():
        t0 = time.perf_counter()
        for i, (ta, b) in enumerate(zip(arrivals, body_of)):
            while True:
                dt = t0 + ta - time.perf_counter()
                if dt <= 0:
                    break
                time.sleep(dt - 0.0002 if dt > 0.0005 else 0)
            cs = bodies[b]
            st, t, _ = srv.submit_ptrs(cs.n, cs.nv, cs.atlas_w, cs.atlas_h, host[b][0], host[b][1],
                                       np.empty(cs.n, tabi.PLACEMENT_DTYPE))
            assert st == 0
            tickets[i] = t
            ready.release()

    def collector():
        for i in range(len(arrivals)):
            ready.acquire()
            st, r = srv.wait(tickets[i], 120000)
            assert st == 0
            results[i] = (r.status, r.scale_k, r.t_submit_ns, r.t_start_ns, r.t_done_ns)

    ths = [threading.Thread(target=submitter), threading.Thread(target=collector)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    stats = srv.stats()
    srv.close()
    ok = all(r[0] == 0 and r[1] == ref_k[b] for r, b in zip(results, body_of))
    lat = np.array([(r[4] - r[2]) * 1e-6 for r in results])
    span = (max(r[4] for r in results) - min(r[2] for r in results)) * 1e-9
    nb = stats["batches"] - base["batches"]
    return {
        "value": len(arrivals) / span, "unit": "packs/s",
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "within_15ms": float(np.mean(lat <= 15.0)), "budget_ms": 15.0,
        "requests": len(arrivals), "rate_per_s": args.serve_rate, "seconds": args.serve_seconds,
        "distinct_bodies": len(bodies), "charts_mean": float(np.mean([bodies[b].n for b in body_of])),
        "lanes": args.serve_lanes, "scale_fanout": args.serve_fanout, "arena_bytes": 8 << 30,
        "batches": nb, "mean_batch": (stats["launched"] - base["launched"]) / max(1, nb),
        "max_batch": stats["max_batch"], "results_equal_alone": ok,
        "plain_fifo": {"value": len(arrivals) / plain_span, "unit": "packs/s",
                       "p50_ms": float(np.percentile(plain_lat, 50)),
                       "p99_ms": float(np.percentile(plain_lat, 99)),
                       "within_15ms": float(np.mean(plain_lat <= 15.0)),
                       "how": "the single-atlas packer serving the same arrivals one at a time (FIFO), "
                              "from each body's measured tabi_pack_device time"},
        "how": "tabi_server: 8 GiB arena over the lanes, continuous batching; one submitting thread at the "
               "arrival times, one collecting thread; latency = result handed over - submitted",
    }


def run_reference(args, rank, world):
    """The CPU oracle on the same atlases: one atlas per step, in batch order."""
    import oracle
    if rank != 0:
        return None
    sets = workload(max(1, min(args.atlases, args.warmup + args.steps)))
    oracle.build()
    for i in range(args.warmup):
        oracle.pack(sets[i % len(sets)])
    times = []
    for i in range(args.steps):
        cs = sets[(args.warmup + i) % len(sets)]
        t0 = time.perf_counter()
        r = oracle.pack(cs)
        times.append(time.perf_counter() - t0)
        assert r.status == 0
    tot = float(np.sum(times))
    v = args.steps / tot
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "packs/s", "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "p50_ms": 1e3 * float(np.percentile(times, 50)), "p99_ms": 1e3 * float(np.percentile(times, 99)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64 (integer path)",
        "data": "synthetic (seeded star charts)",
        "config": {"workload": WORKLOAD, "atlases_sampled": args.steps, "candidates": 64,
                   "step": "one atlas of the batch, in batch order"},
        "cpu_baseline": {"value": v, "unit": "packs/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} atlases of the batch, one per step, one host core"},
        "e2e": {"value": v, "unit": "packs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res))
        return
    sets = workload(args.atlases)  # spawned generator pool, before any CUDA work
    served_inputs = None if args.no_serve or rank != 0 else serve_workload(args)
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    res = run_ours(args, rank, world, local, sets)
    if served_inputs is not None:
        res["served"] = run_served(args, local, *served_inputs)
    if rank == 0:
        if not args.no_cpu_baseline:
            res["cpu_baseline"] = cpu_baseline(sets)
        print(json.dumps(res))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
