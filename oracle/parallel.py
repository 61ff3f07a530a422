"""The oracle's scale search spread over host cores (test and baseline
infrastructure, like the rest of ``oracle``).

``pack()`` tries the candidates S = 16j one after another from the top.
Candidates are independent (Sec. 3.1: the paper gives each its own work
group), so this driver evaluates them in waves of ``width`` candidates, one
``pack_scale`` per process of a spawned pool, and then walks each wave's
results in the same descending order and with the same stopping and
choice rule as ``pack()`` (the area-weighted scale sum of Sec. 4.4, ties
keeping the larger S).  The result is the sequential oracle's; only the
order of evaluation differs.
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np

from . import chart_area2, default_params, pack_scale, prep, sort


def _scale(job):
    rec, perm, W, H, k, params = job
    ok, place, stats = pack_scale(rec, perm, W, H, k, params)
    return ok, place, stats


def pool(workers: int | None = None):
    """A pool of spawned processes (safe to start after CUDA is initialised)."""
    workers = workers or (os.cpu_count() or 1)
    return cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))


def pack_parallel(cs, ex, width: int, params=None):
    """(status, S, place[n, 7] of the chosen candidate in sorted order, perm):
    ``pack()``'s result with ``width`` candidates evaluated at a time on the
    pool ``ex``.  status 0 ok, 2 no fit."""
    params = default_params() if params is None else params
    rec = prep(cs, params)
    perm = sort(rec)
    area = chart_area2(cs)[perm].astype(object)
    area_total = int(area.sum())
    best_k, best_score, best_place = 0, 0, None
    j = 64
    while j >= 1:
        if best_k and 16 * j * area_total <= best_score:
            break
        js = list(range(j, max(0, j - width), -1))
        res = list(ex.map(_scale, [(rec, perm, cs.atlas_w, cs.atlas_h, 16 * jj, params) for jj in js]))
        for jj, (ok, place, _) in zip(js, res):
            k = 16 * jj
            if best_k and k * area_total <= best_score:
                j = 0
                break
            if not ok:
                continue
            score = int((area * place[:, 6].astype(object)).sum())
            if not best_k or score > best_score:
                best_k, best_score, best_place = k, score, place
        else:
            j -= width
    return (0 if best_k else 2), best_k, best_place, perm
