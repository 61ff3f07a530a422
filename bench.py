"""Benchmark of the GB300 atlas packer: the batched and the served forms
against the plain single-atlas packer.

Batched (one step): 256 independent atlases (chart counts uniform in
50..5,000, atlas sides drawn from 1024/2048/4096, star-shaped charts with
6-64 vertices, log-normal areas sigma 1.0, aspect 1:1-1:8), packed together
by one launch sequence replayed from a captured CUDA graph, 1-px gutters, 64
candidate scales per atlas: every stage of the hot path (prep, sort,
envelope raster, compaction, row loop, tail, selection) for all 256
atlases.  The launch shape is autotuned once before timing (tabi_autotune;
no knob changes a result).

Prints one JSON line.  value: atlases packed per second, inputs resident in
HBM, L2 flushed (256 MiB write on the packing stream) before every step,
each step bracketed by CUDA events on the packing stream.  e2e: the same
batch through the host-buffer entry point (tabi_pack_batch) from pinned host
memory, the host<->device copies inside the timed region.  plain: the same
atlases through the single-atlas entry point, one call each; configs: the
three single-atlas workloads (64 charts on 512^2, 2,000 stars on 2048^2,
20,000 Pareto charts on 4096^2) through the plain packer.

served: the serving loop (tabi_server, continuous batching, 8 GiB arena,
the overlap counter behind every result) under the Poisson stream of 2,000
requests/s for 10 s (20,018 requests, chart counts log-uniform 16..20,000,
sides 512..4096, every body distinct, seeded and cached with its SHA-256),
beside the plain packer serving the same arrivals in real time one request
at a time; both again with the arrival times rescaled to 1,000, 4,000 and
8,000 requests/s, and the rate at which each one's p99 crosses the 15 ms
budget.  The roofline stage times come from CUDA events the library records
on the packing stream around every stage, over K further steps.

cpu_baseline: the CPU oracle single-threaded and with its candidates spread
over every host core, on the three single-atlas workloads and on the
batch's atlases.  --impl reference times the CPU oracle on the batch's
atlases one per step.

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
    ap.add_argument("--no-configs", action="store_true", help="skip the single-atlas workloads")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="the stream's own arrival rate")
    ap.add_argument("--serve-rates", default="1000,2000,4000,8000",
                    help="rates the same stream is replayed at (arrival times rescaled)")
    ap.add_argument("--serve-requests", type=int, default=0, help="first N requests of the stream (0: all)")
    ap.add_argument("--serve-lanes", type=int, default=4)
    ap.add_argument("--serve-fanout", type=int, default=8)
    ap.add_argument("--cpu-budget", type=float, default=8.0,
                    help="seconds of oracle time per baseline leg on the batch's atlases")
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


def host_info() -> dict:
    """Host cores and CPU model (lscpu, else the platform's name)."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine(),
            "machine": platform.machine()}


def cpu_baseline(sets, singles, budget_s: float):
    """The CPU oracle as it stands: (a) single-threaded (descending candidates
    with the area-weighted stop), (b) with its candidates evaluated in waves
    of one per host core by a spawned process pool (oracle.parallel; the
    same result).  Each on the single-atlas workloads, then on the batch's
    atlases in order until ``budget_s``.  value = the multi-core rate on the
    batch's atlases."""
    import oracle
    from oracle import parallel
    oracle.build()
    info = host_info()
    P = int(info["nproc"] or 1)
    per = {}
    for name, cs in singles:
        t0 = time.perf_counter()
        r = oracle.pack(cs)
        per[name] = {"charts": cs.n, "k": r.k, "single_ms": round(1e3 * (time.perf_counter() - t0), 3)}
        assert r.status == 0

    def batch_leg(fn):
        t0 = time.perf_counter()
        packs = charts = 0
        ks = []
        for cs in sets:
            ks.append(fn(cs))
            packs += 1
            charts += cs.n
            if time.perf_counter() - t0 > budget_s:
                break
        return packs, charts, time.perf_counter() - t0, ks

    def single(cs):
        r = oracle.pack(cs)
        assert r.status == 0
        return r.k

    n1, c1, t1, k1 = batch_leg(single)
    with parallel.pool(P) as ex:
        parallel.pack_parallel(singles[0][1] if singles else sets[0], ex, P)  # start the workers
        for name, cs in singles:
            t0 = time.perf_counter()
            st, k, _, _ = parallel.pack_parallel(cs, ex, P)
            per[name]["multi_ms"] = round(1e3 * (time.perf_counter() - t0), 3)
            assert st == 0 and k == per[name]["k"]

        def multi(cs):
            st, k, _, _ = parallel.pack_parallel(cs, ex, P)
            assert st == 0
            return k
        nP, cP, tP, kP = batch_leg(multi)
    m = min(len(k1), len(kP))
    assert k1[:m] == kP[:m]
    return {"value": nP / tP, "unit": "packs/s", "cores": P, "kind": "oracle",
            "sample": (f"the first {nP} atlases of the batch ({cP} charts), {tP:.1f} s, candidates in waves of "
                       f"{P} over a spawned pool of {P} processes"),
            "host": info,
            "single_thread": {"value": n1 / t1, "unit": "packs/s", "cores": 1,
                              "sample": f"the first {n1} atlases of the batch ({c1} charts), {t1:.1f} s"},
            "configs": per}


# DRAM read + write of every raster_kernel launch of one batch of this
# workload (ncu, direct launches, the launch shape below), with a digest of
# the kernel's sources at capture time; the bench reports it per launch
# while the sources and the shape match, else null.
RASTER_NCU = {"dram_bytes_per_step": 2720220160, "sources_sha256_16": "43b3a91043a33beb",
              "shape": {"scale_fanout": 2, "chunks": 4, "progressive_bound": 1},
              "profile": "ncu capture of this workload's raster launches (profiles/raster_kernel_batch256.md)"}


def raster_sources_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("raster.cu", "raster_math.cuh", "raster_dev.cuh"):
        with open(os.path.join(ROOT, "paper_2602_07782_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def raster_ops_per_word(g: int) -> int:
    """Integer operations one padded scanline word of an envelope needs by
    its definition (App. A proxies, Sec. 4.1.1 merge, Sec. 5 gutter): the
    ten local-AABB slices of the scanline's own axis and the ten of the
    other axis, each a subtract, an unsigned range compare, a min and a
    max (80); the tighter of the two bounds (a max, a min and the guard: 3);
    two OBB bounds, each the extreme of two lines (a multiply-add and an
    exact division by multiply-high, shift and subtract per line, then a
    max or min: 9) and the corner override (two compares and a select: 3)
    (24); the combination with the slices and the clamps to the chart box
    (6); the gutter dilation, a min and a max per neighbour over 2g
    neighbours (4g); packing the word and the deepest bottom (3)."""
    return 80 + 3 + 24 + 6 + 4 * g + 3


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
    """Unavoidable HBM bytes of the raster and compaction stages of one batch,
    from the charts' AABBs: the raster writes each evaluated (candidate,
    chart) envelope, 4 B per padded scanline word (Top'/Bot' per column and
    L'/R' per row, two int16 each); the compactor reads the rows once and
    per chart its 16 B of meta, 4 B of offset and writes 4 B of distance and
    1 B of flags."""
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
            for j in js:
                k = 16 * (j + 1)
                wp = ((wq * k + (1 << 18) - 1) >> 18) + 2 * g
                hp = ((hq * k + (1 << 18) - 1) >> 18) + 2 * g
                raster += int(4 * (wp.sum() + hp.sum()))
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


def run_ours(args, rank, world, local, sets, singles):
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
    cfg_res = plain_configs(tabi, torch, ctx, dev, stream, flush, singles, args.warmup) if singles else None

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
    # the raster's algorithmic bytes: 4 B per padded scanline word it
    # writes (Top'/Bot' or L'/R', two int16)
    alg["raster"] = 4 * raster_words
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
    # traffic per launch: the captured launches' DRAM bytes per step over
    # the launches of a step, while the kernel and the shape are unchanged
    traffic = None
    if (RASTER_NCU and dom == "raster" and raster_sources_digest() == RASTER_NCU["sources_sha256_16"]
            and all(tuning.get(k) == v for k, v in RASTER_NCU["shape"].items())):
        traffic = int(RASTER_NCU["dram_bytes_per_step"] / launches_dom)
    hbm_view = {"kernel": dom, "bound": "hbm", "achieved": round(achieved_gbs, 2), "peak": hbm_peak,
                "unit": "GB/s", "frac": round(achieved_gbs / hbm_peak, 5), "traffic": traffic,
                "traffic_source": (RASTER_NCU["profile"] if traffic else
                                   "null: no ncu capture of the current kernel at this launch shape"),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": int(dom_bytes), "bytes_per_word": 4 if dom == "raster" else None,
                "avg_launch_ms": round(dom_ms, 4), "launches_per_step": int(launches_dom)}
    roofline = hbm_view
    if dom == "raster":
        # the raster is bound by integer issue (ncu: ALU pipe and issue slots
        # busiest, DRAM far from peak): algorithmic integer operations per
        # launch over its average event-timed launch, against the measured
        # rate of the same operation mix on this GPU
        int_rate = tabi.measure_int_rate(local)
        ops_launch = raster_words * raster_ops_per_word(1) / launches_dom
        achieved_t = ops_launch / (dom_ms * 1e-3) / 1e12 if dom_ms > 0 else 0.0
        roofline = {"kernel": "raster", "bound": "alu", "achieved": round(achieved_t, 4),
                    "peak": round(int_rate / 1e12, 3), "unit": "Tops/s",
                    "frac": round(achieved_t / (int_rate / 1e12), 5), "traffic": traffic,
                    "traffic_source": hbm_view["traffic_source"],
                    "peak_source": ("measured: tabi_measure_int_rate, the rate of the raster's 32-bit integer "
                                    "mix (add, min, max, multiply-high, xor, compare-select, subtract) over "
                                    "all SMs, CUDA events, best of five"),
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
        "configs": cfg_res,
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


def single_atlas_configs():
    """The three single-atlas workloads: 64 convex/L/U charts on 512^2,
    2,000 stars on 2048^2, 20,000 Pareto-sized charts with strips and deep
    concavities on 4096^2."""
    import synth
    return [("C1_plain64", synth.plain64()), ("C2_stars2k", synth.stars2k()), ("C3_pareto20k", synth.pareto20k())]


def plain_configs(tabi, torch, ctx, dev, stream, flush, singles, warm, reps=10):
    """Each single-atlas workload through the plain packer: tabi_pack_device
    (inputs resident) and tabi_pack (host buffers, copies inside), L2 flushed
    before every call, wall clock around the stream-synchronous call."""
    params = tabi.params_default()
    out = {}
    for name, cs in singles:
        keep, _ = device_requests(tabi, torch, dev, [cs])
        offs, verts, o = keep[0]
        dts, hts, ks = [], [], set()
        for r in range(warm + reps):
            with torch.cuda.stream(stream):
                flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, k = ctx.pack_device(cs.n, cs.nv, cs.atlas_w, cs.atlas_h, offs, verts, o, params, stream=stream)
            dt = time.perf_counter() - t0
            assert st == 0, ctx.last_error()
            ks.add(k)
            if r >= warm:
                dts.append(1e3 * dt)
        hout = np.zeros(cs.n, tabi.PLACEMENT_DTYPE)
        for r in range(warm + reps):
            with torch.cuda.stream(stream):
                flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = ctx.pack(cs, params, stream=stream, out=hout)
            dt = time.perf_counter() - t0
            assert res.status == 0
            ks.add(res.k)
            if r >= warm:
                hts.append(1e3 * dt)
        assert len(ks) == 1
        dts, hts = np.array(dts), np.array(hts)
        out[name] = {"charts": cs.n, "vertices": cs.nv, "atlas": [cs.atlas_w, cs.atlas_h], "k": ks.pop(),
                     "p50_ms": round(float(np.percentile(dts, 50)), 4), "p99_ms": round(float(np.percentile(dts, 99)), 4),
                     "packs_per_s": round(1e3 / float(dts.mean()), 2),
                     "host_entry_p50_ms": round(float(np.percentile(hts, 50)), 4),
                     "host_entry_p99_ms": round(float(np.percentile(hts, 99)), 4)}
    out["how"] = (f"plain single-atlas packer, {reps} calls each after {warm} warm-up calls, L2 flushed before "
                  "each; p50/p99 of tabi_pack_device (inputs in HBM) and of tabi_pack (host buffers)")
    return out


def serve_workload(args):
    """The served stream: Poisson arrivals at --serve-rate for
    --serve-seconds, every request's body distinct (synth fixtures, cached
    with their SHA-256; the first --serve-requests if given)."""
    import synth
    st = synth.serve_stream_fixtures(rate=args.serve_rate, duration=args.serve_seconds)
    if args.serve_requests:
        st.arrivals = st.arrivals[:args.serve_requests]
        st.bodies = st.bodies[:args.serve_requests]
        st.seeds = st.seeds[:args.serve_requests]
    return st


def _sleep_until(t: float):
    while True:
        dt = t - time.perf_counter()
        if dt <= 0:
            return
        time.sleep(dt - 0.0002 if dt > 0.0005 else 0)


def _lat_summary(lat_ms, span_s, R):
    return {"value": R / span_s, "unit": "packs/s", "p50_ms": float(np.percentile(lat_ms, 50)),
            "p99_ms": float(np.percentile(lat_ms, 99)), "max_ms": float(lat_ms.max()),
            "within_15ms": float(np.mean(lat_ms <= 15.0))}


def served_run(tabi, srv, arrivals, bodies, out_all, first):
    """The stream through tabi_server: one thread submits each request at
    its arrival time, another waits for the results in order.  Latency =
    (submit call - scheduled arrival) + (result handed over - submitted,
    the library's clock).  Placements land in out_all at first[i]."""
    R = len(arrivals)
    lag = np.zeros(R)
    tickets = [None] * R
    k = np.zeros(R, np.int32)
    lat = np.zeros(R)
    sub = np.zeros(R, np.int64)
    done = np.zeros(R, np.int64)
    qual = np.zeros((R, 3), np.int64)
    bad = []
    ready = threading.Semaphore(0)

    def submitter():
        t0 = time.perf_counter()
        for i in range(R):
            _sleep_until(t0 + arrivals[i])
            lag[i] = time.perf_counter() - (t0 + arrivals[i])
            cs = bodies[i]
            out = out_all[first[i]:first[i] + cs.n]
            st, t, _ = srv.submit_ptrs(cs.n, cs.nv, cs.atlas_w, cs.atlas_h, cs.offsets, cs.verts, out)
            tickets[i] = t if st == 0 else None
            ready.release()

    def collector():
        for i in range(R):
            ready.acquire()
            if tickets[i] is None:
                bad.append((i, "submit"))
                continue
            st, r = srv.wait(tickets[i], 120000)
            if st != 0 or r.status != 0:
                bad.append((i, st, r.status))
                continue
            k[i] = r.scale_k
            sub[i], done[i] = r.t_submit_ns, r.t_done_ns
            lat[i] = 1e3 * lag[i] + 1e-6 * (r.t_done_ns - r.t_submit_ns)
            qual[i] = (r.overlap_texels, r.gutter_texels, r.outside_texels)

    ths = [threading.Thread(target=submitter), threading.Thread(target=collector)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    assert not bad, f"served requests failed: {bad[:5]}"
    span = 1e-9 * (done.max() - sub.min()) + lag[0]
    return lat, span, k, qual


def plain_run(tabi, ctx, params, arrivals, bodies, out_all, first):
    """The same arrivals through the plain packer (tabi_pack, host buffers,
    one request at a time, in arrival order, in real time).  Latency =
    finished - scheduled arrival; service = finished - started."""
    R = len(arrivals)
    k = np.zeros(R, np.int32)
    lat = np.zeros(R)
    service = np.zeros(R)
    t0 = time.perf_counter()
    for i in range(R):
        ta = t0 + arrivals[i]
        _sleep_until(ta)
        cs = bodies[i]
        out = out_all[first[i]:first[i] + cs.n]
        ts = time.perf_counter()
        st, k[i] = ctx.pack_host_ptrs(cs.n, cs.nv, cs.atlas_w, cs.atlas_h, cs.offsets.ctypes.data,
                                      cs.verts.ctypes.data, out.ctypes.data, params)
        te = time.perf_counter()
        assert st == 0, ctx.last_error()
        lat[i] = 1e3 * (te - ta)
        service[i] = te - ts
    span = time.perf_counter() - (t0 + arrivals[0])
    return lat, span, k, service


def crossing(points, budget=15.0):
    """Rate at which p99 first exceeds the budget, interpolated linearly in
    p99 over log(rate) between the bracketing measured rates."""
    pts = sorted(points)
    if pts[0][1] > budget:
        return {"rate": None, "note": f"above the budget already at {pts[0][0]:g}/s"}
    for (r1, p1), (r2, p2) in zip(pts, pts[1:]):
        if p2 > budget >= p1:
            f = (budget - p1) / (p2 - p1)
            return {"rate": round(float(np.exp(np.log(r1) + f * (np.log(r2) - np.log(r1)))), 1),
                    "between": [r1, r2]}
    return {"rate": None, "note": f"within the budget up to {pts[-1][0]:g}/s"}


def run_served(args, local, stream):
    """The served stream and the plain packer on the same arrivals, at the
    stream's own rate and replayed at --serve-rates (arrival times
    rescaled), plus a burst (every request at once)."""
    import torch

    from paper_2602_07782_gb300 import tabi
    torch.cuda.set_device(local)
    bodies = stream.bodies
    R = len(bodies)
    ns = np.array([cs.n for cs in bodies], np.int64)
    first = np.zeros(R + 1, np.int64)
    np.cumsum(ns, out=first[1:])
    ref = np.zeros(int(first[-1]), tabi.PLACEMENT_DTYPE)   # the plain packer's placements (alone)
    buf = np.zeros(int(first[-1]), tabi.PLACEMENT_DTYPE)   # the run being compared with it
    big = list(np.argsort(-np.array([cs.nv for cs in bodies]))[:48]) + list(range(16))

    ctx = tabi.Context(arena_bytes=8 << 30, device=local)
    params = tabi.params_default()
    # warm-up: graphs of the launch shapes the stream needs (every tenth
    # body and the largest), staging
    for b in sorted(set(big) | set(range(0, R, 10))):
        cs = bodies[b]
        o = buf[first[b]:first[b] + cs.n]
        st, _ = ctx.pack_host_ptrs(cs.n, cs.nv, cs.atlas_w, cs.atlas_h, cs.offsets.ctypes.data,
                                   cs.verts.ctypes.data, o.ctypes.data, params)
        assert st == 0, ctx.last_error()
    sp = tabi.params_default(scale_fanout=args.serve_fanout)
    srv = tabi.Server(lanes=args.serve_lanes, max_batch=64, arena_bytes=8 << 30, params=sp, check=1)
    # warm-up: the largest bodies, all at once and twice, so that every
    # lane has grown its pinned staging to a full batch of large requests
    # before the timed runs (a first growth costs a pinned allocation)
    largest = list(np.argsort(-np.array([cs.nv for cs in bodies]))[:256])
    # and the whole stream once at the stream's own rate, untimed, so the
    # graph of every launch shape it meets is captured before the timed runs
    served_run(tabi, srv, stream.arrivals, bodies, buf, first)
    for _ in range(2):
        tickets = []
        for b in largest:
            cs = bodies[b]
            st, t, _ = srv.submit_ptrs(cs.n, cs.nv, cs.atlas_w, cs.atlas_h, cs.offsets, cs.verts,
                                       buf[first[b]:first[b] + cs.n])
            assert st == 0
            tickets.append(t)
        for t in tickets:
            st, r = srv.wait(t, 120000)
            assert st == 0 and r.status == 0

    base_rate = args.serve_rate
    rates = sorted({float(x) for x in args.serve_rates.split(",") if x} | {base_rate})
    sweep = []
    equal = True
    k_ref = None
    plain_service = None
    head = None
    for rate in rates:
        arr = stream.arrivals * (base_rate / rate)
        if k_ref is None:
            lat_p, span_p, k_ref, plain_service = plain_run(tabi, ctx, params, arr, bodies, ref, first)
        else:
            lat_p, span_p, kp, _ = plain_run(tabi, ctx, params, arr, bodies, buf, first)
            equal &= bool(np.array_equal(kp, k_ref)) and bool(np.array_equal(buf, ref))
        s0 = srv.stats()
        lat_s, span_s, ks, qual = served_run(tabi, srv, arr, bodies, buf, first)
        s1 = srv.stats()
        equal &= bool(np.array_equal(ks, k_ref)) and bool(np.array_equal(buf, ref))
        nb = s1["batches"] - s0["batches"]
        pt = {"rate_per_s": rate,
              "served": dict(_lat_summary(lat_s, span_s, R), batches=nb,
                             mean_batch=(s1["launched"] - s0["launched"]) / max(1, nb)),
              "plain": _lat_summary(lat_p, span_p, R),
              "check": {"checked": s1["checked"] - s0["checked"],
                        "violations": s1["check_violations"] - s0["check_violations"],
                        "device_ms_total": 1e-6 * (s1["check_ns"] - s0["check_ns"]),
                        "counts_nonzero": int(np.count_nonzero(qual))}}
        sweep.append(pt)
        if rate == base_rate:
            head = pt
    # burst: every request at time 0
    s0 = srv.stats()
    lat_b, span_b, kb, _ = served_run(tabi, srv, np.zeros(R), bodies, buf, first)
    s1 = srv.stats()
    equal &= bool(np.array_equal(kb, k_ref)) and bool(np.array_equal(buf, ref))
    nb = s1["batches"] - s0["batches"]
    stats = srv.stats()
    srv.close()
    ctx.close()
    checked = sum(p["check"]["checked"] for p in sweep)
    viol = sum(p["check"]["violations"] for p in sweep)
    check_ms = sum(p["check"]["device_ms_total"] for p in sweep)
    return {
        **{k_: head["served"][k_] for k_ in ("value", "unit", "p50_ms", "p99_ms", "max_ms", "within_15ms")},
        "budget_ms": 15.0, "rate_per_s": base_rate, "seconds": args.serve_seconds, "requests": R,
        "distinct_bodies": int(np.unique(stream.seeds).size),
        "charts_mean": float(ns.mean()), "charts_total": int(ns.sum()),
        "vertices_total": int(sum(cs.nv for cs in bodies)),
        "fixtures": {"sha256": stream.sha256, "generator": "synth.stars_fast over synth.serve_specs",
                     "key": stream.key, "generated_s": round(stream.generated_s, 1)},
        "lanes": args.serve_lanes, "scale_fanout": args.serve_fanout, "arena_bytes": 8 << 30,
        "batches": head["served"]["batches"], "mean_batch": head["served"]["mean_batch"],
        "max_batch": stats["max_batch"],
        "results_equal_alone": equal,
        "compared": ("the scale and every placement of every request, at every rate and in the burst, "
                     "against the plain packer's result for the request alone"),
        "check": {"on_every_result": True, "checked": checked, "violations": viol,
                  "mean_us_per_result": round(1e3 * check_ms / max(1, checked), 2),
                  "how": "overlap and gutter counter on the device behind every served batch "
                         "(inside the served latency)"},
        "plain": dict(head["plain"], capacity_packs_per_s=R / float(plain_service.sum()),
                      how="measured: tabi_pack with host buffers, the same arrivals in real time, one request "
                          "at a time in arrival order; latency = finished - scheduled arrival"),
        "sweep": sweep,
        "burst": {"served": dict(_lat_summary(lat_b, span_b, R), batches=nb,
                                 mean_batch=(s1["launched"] - s0["launched"]) / max(1, nb)),
                  "plain_capacity_packs_per_s": R / float(plain_service.sum()),
                  "how": "every request submitted at once; plain capacity = requests / summed service time"},
        "p99_crosses_15ms": {"served": crossing([(p["rate_per_s"], p["served"]["p99_ms"]) for p in sweep]),
                             "plain": crossing([(p["rate_per_s"], p["plain"]["p99_ms"]) for p in sweep])},
        "how": "tabi_server: 8 GiB arena over the lanes, continuous batching, the overlap counter on; one "
               "submitting thread at the arrival times, one collecting thread",
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
                         "sample": f"{args.steps} atlases of the batch, one per step, one host core",
                         "host": host_info()},
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
    singles = [] if args.no_configs or rank != 0 else single_atlas_configs()
    served_inputs = None if args.no_serve or rank != 0 else serve_workload(args)
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    res = run_ours(args, rank, world, local, sets, singles)
    if served_inputs is not None:
        res["served"] = run_served(args, local, served_inputs)
    if rank == 0:
        if not args.no_cpu_baseline:
            res["cpu_baseline"] = cpu_baseline(sets, singles, args.cpu_budget)
        print(json.dumps(res))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
