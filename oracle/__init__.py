"""CPU oracle for the TABI packing path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``tabi_oracle.c`` (plain
sequential C, compiled with gcc) through ctypes and shares nothing with the
CUDA path except the seeded inputs from ``synth``.

Functions follow the paper's steps (Gu, Vining, Sheffer, arXiv 2602.07782):
``prep`` (Sec. 3.1, Sec. 4.1.1, App. A), ``sort`` (Sec. 3.1),
``envelope``/``envelope_padded`` (App. A "Parallel Pushing Algorithm",
Sec. 4.1.1 merge, Sec. 5 gutters), ``hcompact`` (Sec. 4.1.2, App. A
interlock), ``pack_scale`` (Algorithms 2-5, Sec. 4.2, the prefix-sum tail of
Sec. 4.4) and ``pack`` (the scale search, Sec. 3.1 / Sec. 5, with Sec. 4.4's
area-weighted choice).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tabi_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "libtabi_oracle.so")

K = 10  # local AABBs per axis by default (App. A); the slots of a record hold up to 10
REC = 128
# record field offsets (mirror of the enum in tabi_oracle.c)
R = dict(ORIG=0, MINX=1, MINY=2, W0=3, H0=4, WQ=5, HQ=6, ROT=7, FLIPY=8, FLIPX=9,
         OBBM=10, U0=11, U1=12, V0=13, V1=14, X=15, Y=26, YLO=37, YHI=47, XLO=57,
         XHI=67, ATOP=77, ABOT=78, ALEFT=79, ARIGHT=80, ABL2=81, ABR2=82, LK=83)

F_HC, F_BALANCE, F_OBB, F_LAABB = 1, 2, 4, 8
F_ALL = F_HC | F_BALANCE | F_OBB | F_LAABB


def default_params(gutter=1, knee_abs=10, knee_rel=20, lr_sig=10, knee_margin=1, flags=F_ALL, laabb_k=K,
                   topt=10, hybrid_min=10000):
    """Paper defaults: 1-px gutter (Sec. 5), knee thresholds 10 % / 20 % and
    the 10 % left/right significance (App. A), knee margin 1 texel, K = 10
    local AABBs per axis (App. A; Tab. 13 ablates 2 and 5, the oracle takes
    any K in 1..10), prefix-sum folding past t_opt = 1 % of the atlas height
    (``topt`` in permille; 0 = off) for atlases of more than 10,000 charts
    (Sec. 4.4, Tab. 4)."""
    return np.array([gutter, knee_abs, knee_rel, lr_sig, knee_margin, flags, laabb_k, topt, hybrid_min],
                    np.int32)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no vector intrinsics)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32 = ctypes.c_int32
        _lib.oracle_prep.argtypes = [i32, P, P, P, P]
        _lib.oracle_sort.argtypes = [i32, P, P]
        _lib.oracle_envelope.argtypes = [P, i32, P, P, P, P, P, P, i32]
        _lib.oracle_envelope_padded.argtypes = [P, i32, P, P, P, P, P, P, i32]
        _lib.oracle_hcompact.argtypes = [P, P, i32, P, P]
        _lib.oracle_scale_pairs.argtypes = [i32, P, P, i32, P, P, P, P, P, P]
        _lib.oracle_pack_scale.argtypes = [i32, P, P, i32, i32, i32, P, P, P]
        _lib.oracle_pack.argtypes = [i32, P, P, i32, i32, P, i32, P, P, P, P]
        _lib.oracle_correct_y.argtypes = [i32, i32, P, P, P]
        _lib.oracle_obb_table.argtypes = [P]
        _lib.oracle_chart_area2.argtypes = [i32, P, P, P]
        for f in ("oracle_prep", "oracle_envelope", "oracle_envelope_padded", "oracle_hcompact",
                  "oracle_scale_pairs", "oracle_pack_scale", "oracle_pack"):
            getattr(_lib, f).restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def obb_table():
    out = np.zeros(16, np.int64)
    lib().oracle_obb_table(_p(out))
    return out[:8], out[8:]


def prep(cs, params=None):
    """Per-chart records (input order), int64[n, REC]."""
    params = default_params() if params is None else params
    offs = np.ascontiguousarray(cs.offsets, np.uint32)
    verts = np.ascontiguousarray(cs.verts, np.int32)
    rec = np.zeros((cs.n, REC), np.int64)
    if lib().oracle_prep(cs.n, _p(offs), _p(verts), _p(params), _p(rec)):
        raise ValueError("invalid chart set")
    return rec


def sort(rec):
    n = rec.shape[0]
    perm = np.zeros(n, np.int32)
    lib().oracle_sort(n, _p(np.ascontiguousarray(rec)), _p(perm))
    return perm


@dataclass
class Envelope:
    w: int
    h: int
    top: np.ndarray
    bot: np.ndarray
    left: np.ndarray
    right: np.ndarray


def _env(fn, rec1, k, params, cap):
    rec1 = np.ascontiguousarray(rec1, np.int64)
    wh = np.zeros(2, np.int32)
    bufs = [np.zeros(cap, np.int32) for _ in range(4)]
    rc = fn(_p(rec1), int(k), _p(params), _p(wh), *[_p(b) for b in bufs], cap)
    if rc:
        raise ValueError("envelope larger than buffer")
    w, h = int(wh[0]), int(wh[1])
    return Envelope(w, h, bufs[0][:w].copy(), bufs[1][:w].copy(), bufs[2][:h].copy(), bufs[3][:h].copy())


def envelope(rec1, k, params=None, cap=1 << 15):
    """Unpadded per-column Top/Bot and per-row Left/Right at scale k/1024."""
    params = default_params() if params is None else params
    return _env(lib().oracle_envelope, rec1, k, params, cap)


def envelope_padded(rec1, k, params=None, cap=1 << 15):
    """Gutter-dilated envelope (width w+2g, height h+2g)."""
    params = default_params() if params is None else params
    return _env(lib().oracle_envelope_padded, rec1, k, params, cap)


def hcompact(recA, recB, k, params=None):
    """(d, CannotMoveAbove(A,B), CannotMoveAbove(B,A)) for A left of B."""
    params = default_params() if params is None else params
    out = np.zeros(3, np.int32)
    a = np.ascontiguousarray(recA, np.int64)
    b = np.ascontiguousarray(recB, np.int64)
    if lib().oracle_hcompact(_p(a), _p(b), int(k), _p(params), _p(out)):
        raise ValueError("envelope too large")
    return int(out[0]), int(out[1]), int(out[2])


def scale_pairs(rec, perm, k, params=None):
    """Per sorted position s: d(s,s+1), cannotA(s), cannotB(s), w'_s, h'_s."""
    params = default_params() if params is None else params
    n = rec.shape[0]
    d = np.zeros(n, np.int32)
    ca = np.zeros(n, np.uint8)
    cb = np.zeros(n, np.uint8)
    wp = np.zeros(n, np.int32)
    hp = np.zeros(n, np.int32)
    rc = lib().oracle_scale_pairs(n, _p(np.ascontiguousarray(rec)), _p(np.ascontiguousarray(perm, np.int32)),
                                  int(k), _p(params), _p(d), _p(ca), _p(cb), _p(wp), _p(hp))
    if rc:
        raise ValueError("scale build failed")
    return d, ca, cb, wp, hp


def pack_scale(rec, perm, W, H, k, params=None):
    """Algorithm 5 at one scale.  Returns (success, place[n,7] in sorted order
    (x, y, mirror, row, compacting on, fold: 0 atlas width, 1 knee, 2 prefix-sum
    tail, the chart's scale: k, or the tail's k'), stats[8]: rows, knee-folded
    rows, knees found, final max frontline, charts placed, tail rows, the
    tail's scale k' (0: none), first tail chart (n: none))."""
    params = default_params() if params is None else params
    n = rec.shape[0]
    place = np.full((n, 7), -1, np.int32)
    stats = np.zeros(8, np.int32)
    ok = lib().oracle_pack_scale(n, _p(np.ascontiguousarray(rec)), _p(np.ascontiguousarray(perm, np.int32)),
                                 int(W), int(H), int(k), _p(params), _p(place), _p(stats))
    if ok < 0:
        raise ValueError("scale build failed")
    return bool(ok), place, stats


@dataclass
class PackResult:
    status: int  # 0 ok, 1 invalid, 2 no fit
    k: int       # the chosen candidate S
    place: np.ndarray  # int32[n, 11]: x, y, rot90, flip_x, flip_y, mirror, row, sorted pos, hc, fold, k
    success: np.ndarray | None  # int32[64] per candidate j=1..64 (k=16j) if all_scales
    stats: np.ndarray  # int32[8] of the chosen candidate (see pack_scale)
    score: int = 0     # sum over charts of twice the area (Q.8^2) x the chart's scale


def pack(cs, params=None, all_scales=False):
    """The scale search (Sec. 3.1, Sec. 5) with Sec. 4.4's area-weighted
    choice among the successful candidates."""
    params = default_params() if params is None else params
    offs = np.ascontiguousarray(cs.offsets, np.uint32)
    verts = np.ascontiguousarray(cs.verts, np.int32)
    out_k = np.zeros(1, np.int32)
    place = np.full((cs.n, 11), -1, np.int32)
    succ = np.zeros(64, np.int32)
    stats = np.zeros(12, np.int32)
    st = lib().oracle_pack(cs.n, _p(offs), _p(verts), int(cs.atlas_w), int(cs.atlas_h), _p(params),
                           1 if all_scales else 0, _p(out_k), _p(place), _p(succ), _p(stats))
    lo, hi = (int(v) for v in stats[8:12].view(np.int64))
    score = (hi << 64) + (lo & ((1 << 64) - 1))
    return PackResult(int(st), int(out_k[0]), place, succ if all_scales else None, stats[:8].copy(), score)


def chart_area2(cs):
    """Twice the area of every chart's loop (int64, input order): the
    weights of the area-weighted choice in pack()."""
    out = np.zeros(cs.n, np.int64)
    lib().oracle_chart_area2(cs.n, _p(np.ascontiguousarray(cs.offsets, np.uint32)),
                             _p(np.ascontiguousarray(cs.verts, np.int32)), _p(out))
    return out


def _pack_one(args):
    cs, params = args
    r = pack(cs, params)
    return r.status, r.k, r.place


def pack_many(sets, params=None, workers=None):
    """pack() of each chart set, in a pool of spawned processes (spawn keeps
    the pool safe to start after CUDA is initialised).  Returns
    [(status, k, place)]."""
    import concurrent.futures as cf
    import multiprocessing as mp
    params = default_params() if params is None else params
    workers = workers or min(len(sets), os.cpu_count() or 1)
    if workers <= 1:
        return [_pack_one((cs, params)) for cs in sets]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_pack_one, [(cs, params) for cs in sets]))


def correct_y(y, cannotA, cannotB, s0=0, s1=None):
    """Literal Algorithm 2 on int64 offsets y (in place copy returned)."""
    y = np.array(y, np.int64)
    s1 = len(y) - 1 if s1 is None else s1
    ca = np.ascontiguousarray(cannotA, np.uint8)
    cb = np.ascontiguousarray(cannotB, np.uint8)
    lib().oracle_correct_y(int(s0), int(s1), _p(ca), _p(cb), _p(y))
    return y
