"""Exact texel covers of placed charts -- the overlap/gutter metric of the
paper (App. B: texels covered by two or more charts, with and without a
1-pixel gutter dilation), computed independently of the packer.

A texel (c, r) is covered by a chart iff the open square (c, c+1) x (r, r+1)
meets the closed polygon.  Because a simple polygon is the closure of its
interior, that holds iff some polygon edge meets the open square, or the
square's centre lies inside the polygon.  The edge test is the separating
axis test of a closed segment against an open box (axes x, y and the edge
normal), done in exact integer arithmetic.  Coordinates are in units of
2^-18 texel, so a vertex at Q.8 coordinate q drawn at scale k/1024 sits at
q*k.
"""
from __future__ import annotations

import numpy as np

F = 1 << 18


def placed_polygon(verts_q8: np.ndarray, k: int, rot90: int, flip_x: int, flip_y: int,
                   mirror: int) -> tuple[np.ndarray, int, int]:
    """Chart vertices in 2^-18 texel units relative to the chart's box origin,
    following the placement transform: translate the input AABB to the
    origin, rotate (x, y) -> (y, W0 - x) if rot90, reflect y -> Hq - y and
    x -> Wq - x by the orientation flags, scale by k/1024, and reflect
    tx -> w - tx inside the w-texel box when the row ran right to left.
    Returns (int64[nv, 2], w, h)."""
    p = np.asarray(verts_q8, np.int64).reshape(-1, 2)
    mn = p.min(axis=0)
    p = p - mn
    W0, H0 = int(p[:, 0].max()), int(p[:, 1].max())
    if rot90:
        p = np.stack([p[:, 1], W0 - p[:, 0]], axis=1)
    Wq, Hq = int(p[:, 0].max()), int(p[:, 1].max())
    if flip_y:
        p[:, 1] = Hq - p[:, 1]
    if flip_x:
        p[:, 0] = Wq - p[:, 0]
    w = -(-Wq * k // F)
    h = -(-Hq * k // F)
    q = p * k
    if mirror:
        q[:, 0] = w * F - q[:, 0]
    return q, w, h


def cover(poly: np.ndarray, w: int, h: int, margin: int = 0) -> np.ndarray:
    """bool[h + 2*margin, w + 2*margin]: texels (with `margin` extra texels on
    each side) whose open square meets the polygon."""
    poly = np.asarray(poly, np.int64)
    assert np.abs(poly).max(initial=0) < (1 << 31)
    cols = np.arange(-margin, w + margin, dtype=np.int64)
    rows = np.arange(-margin, h + margin, dtype=np.int64)
    a = (cols * F)[None, :]
    b = ((cols + 1) * F)[None, :]
    c = (rows * F)[:, None]
    d = ((rows + 1) * F)[:, None]
    hit = np.zeros((len(rows), len(cols)), bool)
    inside = np.zeros((len(rows), len(cols)), bool)
    # texel centres, doubled to stay integral
    cx2 = (2 * cols + 1) * F
    cy2 = (2 * rows + 1) * F
    n = len(poly)
    for e in range(n):
        x0, y0 = (int(v) for v in poly[e])
        x1, y1 = (int(v) for v in poly[(e + 1) % n])
        if x0 == x1 and y0 == y1:
            continue
        sep = (max(x0, x1) <= a) | (min(x0, x1) >= b) | (max(y0, y1) <= c) | (min(y0, y1) >= d)
        dx, dy = x1 - x0, y1 - y0

        def side(qx, qy):
            return dx * (qy - y0) - dy * (qx - x0)

        s1 = side(a, c)
        s2 = side(b, c)
        s3 = side(a, d)
        s4 = side(b, d)
        allpos = (s1 >= 0) & (s2 >= 0) & (s3 >= 0) & (s4 >= 0)
        allneg = (s1 <= 0) & (s2 <= 0) & (s3 <= 0) & (s4 <= 0)
        hit |= ~(sep | allpos | allneg)
        # crossing number for the doubled centres (half-open rule in y)
        ya, yb = 2 * y0, 2 * y1
        crosses_y = ((ya > cy2) != (yb > cy2))[:, None]
        if y1 != y0:
            # x of the edge at centre height, compared exactly in doubled
            # units: 2*xe = 2*x0 + (2*cy - 2*y0) * dx / dy; centre right of it?
            num = 2 * x0 * dy + (cy2[:, None] - ya) * dx
            lhs = cx2[None, :] * dy
            right_of = (lhs > num) if dy > 0 else (lhs < num)
            inside ^= crosses_y & ~right_of
    return hit | inside


def dilate(mask: np.ndarray, g: int) -> np.ndarray:
    if g == 0:
        return mask.copy()
    out = np.zeros((mask.shape[0] + 2 * g, mask.shape[1] + 2 * g), bool)
    for dy in range(2 * g + 1):
        for dx in range(2 * g + 1):
            out[dy:dy + mask.shape[0], dx:dx + mask.shape[1]] |= mask
    return out


def check_packing(cs, k, place: np.ndarray, gutter: int = 1, envelope_fn=None):
    """Validate a full packing.  `place` is int32[n, >=6] in input order
    (x, y, rot90, flip_x, flip_y, mirror); `k` is the scale of every chart,
    or an array of each chart's scale (the prefix-sum tail of Sec. 4.4 draws
    its charts at a scale of their own).  Returns a dict of violation
    counts: out-of-atlas texels, texels where dilated covers overlap, texels
    where plain covers overlap, and (if envelope_fn(chart, k) is given) cover
    texels outside the chart's own envelope."""
    W, H = cs.atlas_w, cs.atlas_h
    ks = np.broadcast_to(np.asarray(k, np.int64), (cs.n,))
    count = np.zeros((H + 2 * gutter, W + 2 * gutter), np.int16)
    plain = np.zeros((H, W), np.int16)
    out_of_atlas = 0
    outside_env = 0
    for i in range(cs.n):
        x, y, rot, fx, fy, mir = (int(v) for v in place[i, :6])
        poly, w, h = placed_polygon(cs.polygon(i), int(ks[i]), rot, fx, fy, mir)
        cv = cover(poly, w, h)
        if envelope_fn is not None:
            env = envelope_fn(i, int(ks[i]))
            top, bot = env.top, env.bot
            if mir:
                top, bot = top[::-1], bot[::-1]
            rr = np.arange(h)[:, None]
            allowed = (rr >= top[None, :]) & (rr < bot[None, :])
            outside_env += int((cv & ~allowed).sum())
        ys, xs = np.nonzero(cv)
        ax, ay = xs + x, ys + y
        bad = (ax < 0) | (ax >= W) | (ay < 0) | (ay >= H)
        out_of_atlas += int(bad.sum())
        ok = ~bad
        np.add.at(plain, (ay[ok], ax[ok]), 1)
        dv = dilate(cv, gutter)
        ys, xs = np.nonzero(dv)
        ax, ay = xs + x, ys + y  # padded coordinates: shift by -g then +g
        okp = (ax >= 0) & (ax < W + 2 * gutter) & (ay >= 0) & (ay < H + 2 * gutter)
        np.add.at(count, (ay[okp], ax[okp]), 1)
    return dict(out_of_atlas=out_of_atlas,
                gutter_overlap=int((count > 1).sum()),
                overlap=int((plain > 1).sum()),
                outside_envelope=outside_env)
