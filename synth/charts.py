"""Seeded synthetic chart sets for the atlas-packing path.

This module only draws inputs: polygons given as vertex loops in 1/256-texel
fixed point (int32), stored CSR-style (``offsets[n+1]`` into ``verts[2*nv]``,
x/y interleaved), plus the atlas size.  It holds none of the packing method's
arithmetic and is imported by both the CPU oracle tests and the GPU path, so
both sides always see identical inputs.

The workloads stand in for the paper's chart sets (Sec. 5: UV charts and
texture-space-shading charts, 2 to 44,389 charts per atlas, square
power-of-two atlases), which are not available here.  Shapes, size laws and
atlas sizes follow the five workload descriptions used throughout the
project:

* ``plain64``    64 charts, convex (4-16 vertices on an ellipse) or
                 axis-aligned L/U shapes (notch 30-70 %), bounding-box sides
                 uniform 8-128 texels, atlas 512x512.
* ``stars2k``    2,000 star-shaped polygons (6-64 vertices, radii jittered
                 +-40 %), bounding-box areas log-normal (sigma 1.0) with the
                 mean chosen so the summed box area equals the atlas area,
                 aspect ratios log-uniform 1:1-1:8, random orientation,
                 atlas 2048x2048.
* ``pareto20k``  20,000 charts, Pareto(alpha=1.5) box areas scaled so the
                 sum equals the atlas area and truncated at 1 % of it; 10 %
                 long strips (aspect 1:16-1:64), 5 % deep concavities (comb or
                 U, notch >= 60 % of the box), the rest stars; atlas 4096x4096.
* ``batch256``   256 independent atlases, chart counts uniform 50-5,000,
                 atlas sides drawn from {1024, 2048, 4096}, shapes as stars2k.
* ``serve``      a Poisson request stream (rate, duration), chart counts
                 log-uniform 16-20,000, atlas sides from {512,...,4096}.

Every polygon is normalised to an exact integer bounding box of at least one
texel (256 units) per side and then translated by a random offset, so the
packer's own translate step is exercised.  All coordinates stay inside
(-2^20, 2^20).
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass

import numpy as np

Q = 256  # fixed-point units per texel
COORD_LIMIT = 1 << 20


@dataclass
class ChartSet:
    """One packing request: CSR polygons plus the atlas size in texels."""

    offsets: np.ndarray  # uint32[n+1]
    verts: np.ndarray  # int32[2*nv], x0,y0,x1,y1,...
    atlas_w: int
    atlas_h: int
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def nv(self) -> int:
        return int(self.verts.shape[0] // 2)

    def polygon(self, i: int) -> np.ndarray:
        a, b = int(self.offsets[i]), int(self.offsets[i + 1])
        return self.verts[2 * a:2 * b].reshape(-1, 2)


# --------------------------------------------------------------------------
# shape primitives (unit-free float outlines, later normalised to a box)
# --------------------------------------------------------------------------

def _convex(rng, nv):
    ang = np.sort(rng.uniform(0.0, 2.0 * math.pi, nv))
    return np.stack([np.cos(ang), np.sin(ang)], axis=1)


def _star(rng, nv, jitter=0.4):
    base = np.arange(nv) * (2.0 * math.pi / nv)
    ang = base + rng.uniform(-0.3, 0.3, nv) * (2.0 * math.pi / nv)
    rad = 1.0 + rng.uniform(-jitter, jitter, nv)
    return np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)


def _l_shape(rng):
    fx, fy = rng.uniform(0.3, 0.7, 2)
    # unit box with the top-right corner removed
    return np.array([[0, 0], [1 - fx, 0], [1 - fx, fy], [1, fy], [1, 1], [0, 1]], float)


def _u_shape(rng, lo=0.3, hi=0.7):
    fx, fy = rng.uniform(lo, hi, 2)
    a = (1 - fx) / 2
    # unit box with a notch cut from the middle of the top edge
    return np.array([[0, 0], [a, 0], [a, fy], [a + fx, fy], [a + fx, 0], [1, 0],
                     [1, 1], [0, 1]], float)


def _comb(rng):
    teeth = int(rng.integers(2, 5))
    depth = rng.uniform(0.6, 0.85)
    pts = [[0.0, 1.0], [0.0, 0.0]]
    slot = 1.0 / (2 * teeth - 1)
    x = 0.0
    for t in range(teeth):
        x0, x1 = x, x + slot
        pts += [[x0, 0.0], [x1, 0.0]]
        if t < teeth - 1:
            pts += [[x1, depth], [x1 + slot, depth]]
        x = x1 + slot
    pts += [[1.0, 0.0], [1.0, 1.0]]
    out = []
    for p in pts:
        if not out or out[-1] != p:
            out.append(p)
    return np.array(out, float)


def _rotate(pts, theta):
    c, s = math.cos(theta), math.sin(theta)
    return pts @ np.array([[c, s], [-s, c]])


def _to_fixed(pts, box_w, box_h):
    """Map a float outline onto the exact integer box [0,box_w]x[0,box_h]."""
    mn = pts.min(axis=0)
    ext = pts.max(axis=0) - mn
    ext[ext == 0] = 1.0
    u = (pts - mn) / ext
    x = np.rint(u[:, 0] * box_w).astype(np.int64)
    y = np.rint(u[:, 1] * box_h).astype(np.int64)
    q = np.stack([x, y], axis=1)
    keep = np.ones(len(q), bool)
    keep[1:] = np.any(q[1:] != q[:-1], axis=1)
    q = q[keep]
    if len(q) > 1 and np.all(q[0] == q[-1]):
        q = q[:-1]
    if len(q) < 3 or q[:, 0].max() != box_w or q[:, 1].max() != box_h:
        q = np.array([[0, 0], [box_w, 0], [box_w, box_h], [0, box_h]], np.int64)
    return q


def _box_from_area(area_tx, aspect, rng, max_side=4000.0):
    """Texel box (w, h) with w*h = area and h/w = aspect (orientation random)."""
    h = math.sqrt(area_tx * aspect)
    w = area_tx / h
    if rng.random() < 0.5:
        w, h = h, w
    w = min(max(w, 1.0), max_side)
    h = min(max(h, 1.0), max_side)
    return w, h


def _pack(polys, rng, atlas_w, atlas_h, name):
    offs = np.zeros(len(polys) + 1, np.uint32)
    chunks = []
    total = 0
    for i, q in enumerate(polys):
        w = int(q[:, 0].max())
        h = int(q[:, 1].max())
        lim = COORD_LIMIT - 1
        ox = int(rng.integers(-lim // 2, lim - w - lim // 2))
        oy = int(rng.integers(-lim // 2, lim - h - lim // 2))
        qq = q + np.array([ox, oy], np.int64)
        assert np.all(np.abs(qq) < COORD_LIMIT)
        chunks.append(qq.astype(np.int32).reshape(-1))
        total += len(q)
        offs[i + 1] = total
    verts = np.concatenate(chunks) if chunks else np.zeros(0, np.int32)
    return ChartSet(offs, verts.astype(np.int32), atlas_w, atlas_h, name)


def _fixed_side(side_tx):
    return max(Q, int(round(side_tx * Q)))


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def plain64(seed: int = 1, n: int = 64, atlas: int = 512) -> ChartSet:
    rng = np.random.default_rng([seed, 1])
    polys = []
    for _ in range(n):
        bw = rng.uniform(8, 128)
        bh = rng.uniform(8, 128)
        kind = rng.random()
        if kind < 0.5:
            pts = _convex(rng, int(rng.integers(4, 17)))
        elif kind < 0.75:
            pts = _l_shape(rng)
        else:
            pts = _u_shape(rng)
        if rng.random() < 0.5 and kind >= 0.5:
            pts = pts @ np.array([[1, 0], [0, -1]], float)  # mirror: notch at any corner
        polys.append(_to_fixed(pts, _fixed_side(bw), _fixed_side(bh)))
    return _pack(polys, rng, atlas, atlas, f"plain64[{n},{atlas}]")


def _star_chart(rng, area_tx, max_side=4000.0):
    aspect = math.exp(rng.uniform(0.0, math.log(8.0)))
    nv = int(rng.integers(6, 65))
    pts = _star(rng, nv)
    pts[:, 1] *= aspect
    pts = _rotate(pts, rng.uniform(0.0, math.pi))
    ext = pts.max(axis=0) - pts.min(axis=0)
    # box area of the rotated outline follows the drawn area
    s = math.sqrt(area_tx / max(ext[0] * ext[1], 1e-9))
    bw = min(max(ext[0] * s, 1.0), max_side)
    bh = min(max(ext[1] * s, 1.0), max_side)
    return _to_fixed(pts, _fixed_side(bw), _fixed_side(bh))


DENSITY = 4.0  # summed box area / atlas area: puts the best scale near 1/2


def stars(seed: int, n: int, atlas: int, sigma: float = 1.0, density: float = DENSITY) -> ChartSet:
    rng = np.random.default_rng([seed, 2, n, atlas])
    mu = math.log(density * atlas * atlas / n) - sigma * sigma / 2.0
    areas = rng.lognormal(mu, sigma, n)
    polys = [_star_chart(rng, float(a), max_side=min(4000.0, 2.0 * atlas)) for a in areas]
    return _pack(polys, rng, atlas, atlas, f"stars[{n},{atlas}]")


def stars2k(seed: int = 2) -> ChartSet:
    return stars(seed, 2000, 2048)


def _pareto_areas(rng, n, total, cap, alpha=1.5):
    raw = (1.0 - rng.random(n)) ** (-1.0 / alpha)
    lo, hi = 1e-9, total
    for _ in range(100):
        c = math.sqrt(lo * hi) if lo > 0 else hi / 2
        s = np.minimum(raw * c, cap).sum()
        if s > total:
            hi = c
        else:
            lo = c
    return np.maximum(np.minimum(raw * lo, cap), 1.0)


def pareto20k(seed: int = 3, n: int = 20000, atlas: int = 4096,
              density: float = DENSITY) -> ChartSet:
    rng = np.random.default_rng([seed, 3, n, atlas])
    areas = _pareto_areas(rng, n, density * atlas * atlas, 0.01 * atlas * atlas)
    polys = []
    for a in areas:
        u = rng.random()
        if u < 0.10:  # long thin strip
            aspect = rng.uniform(16.0, 64.0)
            bw, bh = _box_from_area(float(a), aspect, rng)
            if rng.random() < 0.5:
                pts = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
            else:
                pts = _star(rng, int(rng.integers(6, 17)), 0.15)
            polys.append(_to_fixed(pts, _fixed_side(bw), _fixed_side(bh)))
        elif u < 0.15:  # deep concavity
            bw, bh = _box_from_area(float(a), math.exp(rng.uniform(0, math.log(4.0))), rng)
            pts = _comb(rng) if rng.random() < 0.5 else _u_shape(rng, 0.6, 0.85)
            if rng.random() < 0.5:
                pts = pts @ np.array([[1, 0], [0, -1]], float)
            polys.append(_to_fixed(pts, _fixed_side(bw), _fixed_side(bh)))
        else:
            polys.append(_star_chart(rng, float(a)))
    return _pack(polys, rng, atlas, atlas, f"pareto[{n},{atlas}]")


def knees(seed: int, n: int, atlas: int, n_tall: int = 6, density: float = DENSITY) -> ChartSet:
    """Stars plus a few tall charts (30-60 % of the atlas height at full
    scale), so sorted rows contain the sharp height drops ("knees") that the
    balanced folding of Sec. 4.2 reacts to."""
    rng = np.random.default_rng([seed, 7, n, atlas])
    base = stars(seed, n - n_tall, atlas, density=density)
    polys = [base.polygon(i).astype(np.int64) - base.polygon(i).min(axis=0) for i in range(base.n)]
    for _ in range(n_tall):
        h = rng.uniform(0.3, 0.6) * atlas * 2.0
        w = h * rng.uniform(0.15, 0.5)
        pts = _star(rng, int(rng.integers(6, 33)), 0.3) if rng.random() < 0.5 else _l_shape(rng)
        polys.append(_to_fixed(pts, _fixed_side(w), _fixed_side(h)))
    order = rng.permutation(len(polys))
    return _pack([polys[i] for i in order], rng, atlas, atlas, f"knees[{n},{atlas}]")


def batch256_specs(seed: int = 4, count: int = 256, lo: int = 50, hi: int = 5000,
                   sides=(1024, 2048, 4096)) -> list[tuple[int, int, int]]:
    """(chart seed, chart count, atlas side) of each atlas of the batch."""
    rng = np.random.default_rng([seed, 4, count])
    out = []
    for i in range(count):
        n = int(rng.integers(lo, hi + 1))
        side = int(sides[int(rng.integers(0, len(sides)))])
        out.append((seed * 100003 + i, n, side))
    return out


def batch256(seed: int = 4, count: int = 256, lo: int = 50, hi: int = 5000,
             sides=(1024, 2048, 4096)) -> list[ChartSet]:
    return [stars(s, n, side) for s, n, side in batch256_specs(seed, count, lo, hi, sides)]


def _stars_spec(spec):
    return stars(*spec)


def stars_many(specs, workers: int | None = None) -> list[ChartSet]:
    """stars(*spec) for each spec, generated in a pool of spawned processes
    (the same sets as one by one; spawn keeps the pool safe to start after
    CUDA is initialised)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    specs = list(specs)
    workers = workers or min(len(specs), os.cpu_count() or 1)
    if workers <= 1 or len(specs) < 4:
        return [stars(*sp) for sp in specs]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_stars_spec, specs, chunksize=max(1, len(specs) // (4 * workers))))


@dataclass
class Request:
    t_arrive: float  # seconds from stream start
    charts: ChartSet


def serve_specs(seed: int = 5, rate: float = 2000.0, duration: float = 10.0,
                lo: int = 16, hi: int = 20000, sides=(512, 1024, 2048, 4096),
                limit: int | None = None) -> list[tuple[float, int, int, int]]:
    """(arrival time s, chart seed, chart count, atlas side) of each request
    of serve_stream, without generating the charts."""
    rng = np.random.default_rng([seed, 5])
    t = 0.0
    out = []
    i = 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration or (limit is not None and i >= limit):
            break
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        side = int(sides[int(rng.integers(0, len(sides)))])
        out.append((t, seed * 1000003 + i, n, side))
        i += 1
    return out


def serve_stream(seed: int = 5, rate: float = 2000.0, duration: float = 10.0,
                 lo: int = 16, hi: int = 20000, sides=(512, 1024, 2048, 4096),
                 limit: int | None = None) -> list[Request]:
    """Poisson arrivals; chart counts log-uniform in [lo, hi]."""
    return [Request(t, stars(sd, n, side)) for t, sd, n, side in
            serve_specs(seed, rate, duration, lo, hi, sides, limit)]


def rectangles(sizes_tx, atlas_w: int, atlas_h: int, seed: int = 0) -> ChartSet:
    """Axis-aligned rectangles with the given (w, h) in whole texels."""
    rng = np.random.default_rng([seed, 6])
    polys = [np.array([[0, 0], [w * Q, 0], [w * Q, h * Q], [0, h * Q]], np.int64)
             for (w, h) in sizes_tx]
    return _pack(polys, rng, atlas_w, atlas_h, "rects")


def from_polygons(polys_q8, atlas_w: int, atlas_h: int, name: str = "custom") -> ChartSet:
    """Pack explicit int polygons (lists of (x, y) in 1/256 texel) as given."""
    offs = np.zeros(len(polys_q8) + 1, np.uint32)
    chunks = []
    total = 0
    for i, p in enumerate(polys_q8):
        a = np.asarray(p, np.int64).reshape(-1, 2)
        chunks.append(a.astype(np.int32).reshape(-1))
        total += len(a)
        offs[i + 1] = total
    return ChartSet(offs, np.concatenate(chunks).astype(np.int32), atlas_w, atlas_h, name)


WORKLOADS = {
    "plain64": plain64,
    "stars2k": stars2k,
    "pareto20k": pareto20k,
    "knees": knees,
}


# --------------------------------------------------------------------------
# vectorised star sets for the served stream (same shape law as ``stars``,
# drawn with whole-request array operations so that a stream of tens of
# millions of charts is generated in seconds; a different random stream
# from ``stars``, so the sets differ from it chart by chart)
# --------------------------------------------------------------------------

def stars_fast(seed: int, n: int, atlas: int, sigma: float = 1.0, density: float = DENSITY) -> ChartSet:
    """Star-shaped charts as ``stars`` draws them (6-64 vertices, radii
    jittered +-40 %, angular jitter +-30 % of a step, aspect log-uniform
    1:1-1:8, random rotation, log-normal box areas with the summed box
    area ``density`` x the atlas area), every vertex of the set in one
    flat array."""
    rng = np.random.default_rng([seed, 8, n, atlas])
    mu = math.log(density * atlas * atlas / n) - sigma * sigma / 2.0
    area = rng.lognormal(mu, sigma, n)
    aspect = np.exp(rng.uniform(0.0, math.log(8.0), n))
    nv = rng.integers(6, 65, n)
    theta = rng.uniform(0.0, math.pi, n)
    start = np.zeros(n + 1, np.int64)
    np.cumsum(nv, out=start[1:])
    T = int(start[-1])
    seg = np.repeat(np.arange(n), nv)
    idx = np.arange(T) - start[seg]
    step = (2.0 * math.pi) / nv[seg]
    ang = (idx + rng.uniform(-0.3, 0.3, T)) * step
    rad = 1.0 + rng.uniform(-0.4, 0.4, T)
    x0 = rad * np.cos(ang)
    y0 = rad * np.sin(ang) * aspect[seg]
    c, s = np.cos(theta)[seg], np.sin(theta)[seg]
    x = x0 * c - y0 * s
    y = x0 * s + y0 * c
    st = start[:-1]
    mnx, mny = np.minimum.reduceat(x, st), np.minimum.reduceat(y, st)
    exx = np.maximum.reduceat(x, st) - mnx
    exy = np.maximum.reduceat(y, st) - mny
    max_side = min(4000.0, 2.0 * atlas)
    sc = np.sqrt(area / np.maximum(exx * exy, 1e-9))
    box_w = np.maximum(Q, np.rint(np.clip(exx * sc, 1.0, max_side) * Q)).astype(np.int64)
    box_h = np.maximum(Q, np.rint(np.clip(exy * sc, 1.0, max_side) * Q)).astype(np.int64)
    X = np.rint((x - mnx[seg]) / exx[seg] * box_w[seg]).astype(np.int64)
    Y = np.rint((y - mny[seg]) / exy[seg] * box_h[seg]).astype(np.int64)
    keep = np.ones(T, bool)
    keep[1:] = (X[1:] != X[:-1]) | (Y[1:] != Y[:-1])
    keep[st] = True
    cnt = np.add.reduceat(keep.astype(np.int64), st)
    # the last kept vertex of a loop equal to its first closes the loop twice
    pos = np.flatnonzero(keep)
    kst = np.zeros(n + 1, np.int64)
    np.cumsum(cnt, out=kst[1:])
    last = pos[kst[1:] - 1]
    closing = (cnt > 1) & (X[last] == X[st]) & (Y[last] == Y[st])
    keep[last[closing]] = False
    cnt -= closing
    bad = np.flatnonzero(cnt < 3)
    lim = COORD_LIMIT - 1
    ox = rng.integers(-(lim // 2), lim - box_w - lim // 2)
    oy = rng.integers(-(lim // 2), lim - box_h - lim // 2)
    for b in bad:  # degenerate outline (rare): its box instead
        a = int(st[b])
        keep[a:a + int(nv[b])] = False
        keep[a:a + 4] = True
        X[a:a + 4] = (0, box_w[b], box_w[b], 0)
        Y[a:a + 4] = (0, 0, box_h[b], box_h[b])
        cnt[b] = 4
    X += ox[seg]
    Y += oy[seg]
    offs = np.zeros(n + 1, np.uint32)
    verts = np.empty(2 * int(cnt.sum()), np.int32)
    np.cumsum(cnt, out=offs[1:])
    verts[0::2] = X[keep]
    verts[1::2] = Y[keep]
    return ChartSet(offs, verts, atlas, atlas, f"stars_fast[{n},{atlas}]")
