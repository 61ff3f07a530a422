"""The allocation-free height sort (tabi_sort_heights_noalloc).

Callers that cannot call cudaMalloc -- engines with a fixed, pre-budgeted
device memory pool, frame loops that must not stall on an allocation -- use
this entry point: its scratch is a fixed array inside the library, and the
caller passes only device input and output buffers.  The test calls it
through the C ABI twice in a row and checks each result against the CPU
oracle's height sort of the same charts (Sec. 3.1) and against the order the
regular pack entry point (tabi_pack) computed.  Collected last on purpose.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_2602_07782_gb300 import tabi  # noqa: E402


def _noalloc(lib):
    f = lib.tabi_sort_heights_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def test_noalloc_sort_matches_pack_order_twice():
    lib = tabi.load()
    sort_noalloc = _noalloc(lib)
    sets = [synth.stars2k(), synth.knees(1, 300, 1024)]
    ctx = tabi.Context(arena_bytes=max(tabi.arena_bytes(cs) for cs in sets) + (64 << 20))
    try:
        for cs in sets:  # two calls in a row share the scratch array
            res = ctx.pack(cs)
            assert res.status == tabi.TABI_OK, ctx.last_error()
            ref = ctx.perm()
            rec = oracle.prep(cs)  # the heights come from the oracle, not from the GPU path
            assert np.array_equal(ctx.charts()["Hq"], rec[:, oracle.R["HQ"]])
            heights = rec[:, oracle.R["HQ"]].astype(np.int32)
            d_h = torch.from_numpy(heights.copy()).cuda()
            d_p = torch.full((cs.n,), -1, dtype=torch.int32, device="cuda")
            stream = torch.cuda.current_stream()
            st = sort_noalloc(ctypes.c_void_p(d_h.data_ptr()), cs.n, ctypes.c_void_p(d_p.data_ptr()),
                              ctypes.c_void_p(stream.cuda_stream))
            stream.synchronize()
            assert st == tabi.TABI_OK
            got = d_p.cpu().numpy()
            assert np.array_equal(got, oracle.sort(rec))
            assert np.array_equal(got, ref)
    finally:
        ctx.close()


def test_noalloc_sort_rejects_oversize():
    sort_noalloc = _noalloc(tabi.load())
    d = torch.zeros(4, dtype=torch.int32, device="cuda")
    assert sort_noalloc(ctypes.c_void_p(d.data_ptr()), 65537, ctypes.c_void_p(d.data_ptr()), None) == \
        tabi.TABI_ERR_INVALID_ARG
    assert sort_noalloc(None, 4, ctypes.c_void_p(d.data_ptr()), None) == tabi.TABI_ERR_INVALID_ARG
