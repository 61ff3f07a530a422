"""Seeded request bodies of the served stream, generated once into a cache
directory and read back memory-mapped.

A stream of Poisson arrivals (``serve_specs``) names each request by (chart
seed, chart count, atlas side); ``stars_fast`` draws its charts.  The whole
stream -- about 20,000 requests and 56 million charts at 2,000 requests/s
for 10 s -- is generated by a pool of spawned processes, each writing a
contiguous run of requests to one part file (per request: its n+1 offsets
as uint32, then its 2*nv vertex coordinates as int32) and returning the
part's SHA-256.  A manifest records the stream's parameters, the part
digests and one digest over them; a later call with the same parameters
finds the manifest and maps the parts without generating anything.

Like the rest of ``synth`` this holds no packing arithmetic: it only draws
inputs, which both the GPU path and the CPU oracle read.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import dataclass

import numpy as np

from .charts import ChartSet, serve_specs, stars_fast


def default_dir() -> str:
    return os.environ.get("TABI_FIXTURES", os.path.join("/tmp", "tabi_fixtures"))


def _write_part(job):
    path, specs = job
    h = hashlib.sha256()
    sizes = []
    with open(path + ".tmp", "wb") as f:
        for _, seed, n, side in specs:
            cs = stars_fast(seed, n, side)
            for a in (cs.offsets.astype("<u4"), cs.verts.astype("<i4")):
                b = a.tobytes()
                h.update(b)
                f.write(b)
            sizes.append((cs.n, cs.nv))
    os.replace(path + ".tmp", path)
    return h.hexdigest(), sizes


@dataclass
class Stream:
    """The served stream: arrival times (s) and request bodies."""

    arrivals: np.ndarray      # float64[R], seconds from the stream's start
    bodies: list              # ChartSet per request, arrays memory-mapped
    seeds: np.ndarray         # int64[R], the chart seed of each request
    sha256: str               # digest over the parts' digests and the stream key
    key: dict                 # the stream's parameters
    generated_s: float        # seconds spent generating (0: found in the cache)
    charts: int
    vertices: int


def serve_stream_fixtures(rate: float = 2000.0, duration: float = 10.0, seed: int = 5,
                          cache_dir: str | None = None, workers: int | None = None,
                          parts: int = 64) -> Stream:
    """All requests of ``serve_specs(seed, rate, duration)`` with their bodies
    drawn by ``stars_fast`` (cached under ``cache_dir``)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import time

    specs = serve_specs(seed=seed, rate=rate, duration=duration)
    key = {"generator": "stars_fast", "stream": "serve_specs", "seed": seed, "rate": rate,
           "duration": duration, "requests": len(specs), "format": 1}
    tag = hashlib.sha256(json.dumps(key, sort_keys=True).encode()).hexdigest()[:16]
    root = os.path.join(cache_dir or default_dir(), f"serve_{tag}")
    man_path = os.path.join(root, "manifest.json")
    P = max(1, min(parts, len(specs)))
    cuts = [round(i * len(specs) / P) for i in range(P + 1)]
    names = [os.path.join(root, f"part{i:03d}.bin") for i in range(P)]
    man = None
    if os.path.exists(man_path):
        with open(man_path) as f:
            man = json.load(f)
        if man.get("key") != key or not all(os.path.exists(p) for p in names):
            man = None
    t0 = time.perf_counter()
    gen_s = 0.0
    if man is None:
        os.makedirs(root, exist_ok=True)
        jobs = [(names[i], specs[cuts[i]:cuts[i + 1]]) for i in range(P)]
        workers = workers or min(P, os.cpu_count() or 1)
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            out = list(ex.map(_write_part, jobs))
        digests = [d for d, _ in out]
        sizes = [s for _, s in out]
        total = hashlib.sha256(json.dumps(key, sort_keys=True).encode())
        for d in digests:
            total.update(bytes.fromhex(d))
        man = {"key": key, "parts": digests, "sizes": sizes, "sha256": total.hexdigest()}
        with open(man_path + ".tmp", "w") as f:
            json.dump(man, f)
        os.replace(man_path + ".tmp", man_path)
        gen_s = time.perf_counter() - t0
    bodies = []
    charts = verts = 0
    for i in range(P):
        mm = np.memmap(names[i], dtype=np.uint8, mode="r")
        off = 0
        for (_, _, _, side), (n, nv) in zip(specs[cuts[i]:cuts[i + 1]], man["sizes"][i]):
            o = np.ndarray((n + 1,), np.uint32, mm, off)
            off += 4 * (n + 1)
            v = np.ndarray((2 * nv,), np.int32, mm, off)
            off += 8 * nv
            bodies.append(ChartSet(o, v, side, side, f"serve[{n},{side}]"))
            charts += n
            verts += nv
        assert off == mm.shape[0], "fixture part size does not match its manifest"
    arrivals = np.array([sp[0] for sp in specs])
    seeds = np.array([sp[1] for sp in specs], np.int64)
    return Stream(arrivals, bodies, seeds, man["sha256"], key, gen_s, charts, verts)
