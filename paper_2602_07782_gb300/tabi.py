"""Python binding of the GB300 atlas packer (``include/tabi.h``).

Argument marshalling only: every step of the packing path runs in the CUDA
kernels of ``_build/libtabi.so``.  PyTorch provides device memory (the
context arena, device-side inputs and outputs) and streams.  If the library
is missing the import-time loader raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libtabi.so")

TABI_OK, TABI_ERR_INVALID_ARG, TABI_ERR_NO_FIT, TABI_ERR_OOM, TABI_ERR_CUDA, TABI_ERR_TIMEOUT, TABI_ERR_BUSY = range(7)
F_HC, F_BALANCE, F_OBB, F_LAABB = 1, 2, 4, 8
F_ALL = 15
INSPECT_CHARTS, INSPECT_PERM, INSPECT_ENV, INSPECT_ENV_CAP, INSPECT_PAIRS, INSPECT_SCALE = 1, 2, 3, 4, 5, 6
N_SCALES = 64


class Params(ctypes.Structure):
    _fields_ = [("version", ctypes.c_int32), ("gutter", ctypes.c_int32),
                ("knee_abs_pct", ctypes.c_int32), ("knee_rel_pct", ctypes.c_int32),
                ("lr_sig_pct", ctypes.c_int32), ("knee_margin", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("scale_fanout", ctypes.c_int32)]


PLACEMENT_DTYPE = np.dtype([("x", "<i4"), ("y", "<i4"), ("rot90", "u1"), ("flip_x", "u1"),
                            ("flip_y", "u1"), ("mirror", "u1")])

CHART_INFO_DTYPE = np.dtype([
    ("orig", "<i4"), ("Wq", "<i4"), ("Hq", "<i4"), ("rot90", "<i4"), ("flip_y", "<i4"),
    ("flip_x", "<i4"), ("obb_m", "<i4"), ("valid", "<i4"),
    ("u0", "<i8"), ("u1", "<i8"), ("v0", "<i8"), ("v1", "<i8"),
    ("ylo", "<i4", 10), ("yhi", "<i4", 10), ("xlo", "<i4", 10), ("xhi", "<i4", 10),
    ("tlo", "<i4", 10), ("bhi", "<i4", 10), ("llo", "<i4", 10), ("rhi", "<i4", 10),
    ("area_top", "<i8"), ("area_bot", "<i8"), ("area_left", "<i8"), ("area_right", "<i8"),
    ("area_bl2", "<i8"), ("area_br2", "<i8")])

EXPORTS = ["tabi_params_default", "tabi_ctx_create", "tabi_ctx_destroy", "tabi_last_error",
           "tabi_status_str", "tabi_arena_bytes", "tabi_pack", "tabi_pack_device", "tabi_inspect",
           "tabi_stage_times"]
STAGES = ["prep", "sort", "layout", "raster", "hcompact", "rowloop", "select", "pack"]

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA packer library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32 = ctypes.c_int32
    lib.tabi_params_default.argtypes = [P]
    lib.tabi_ctx_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, P, ctypes.c_size_t]
    lib.tabi_ctx_create.restype = ctypes.c_int
    lib.tabi_ctx_destroy.argtypes = [P]
    lib.tabi_last_error.argtypes = [P]
    lib.tabi_last_error.restype = ctypes.c_char_p
    lib.tabi_status_str.argtypes = [ctypes.c_int]
    lib.tabi_status_str.restype = ctypes.c_char_p
    lib.tabi_arena_bytes.argtypes = [i32, i32, i32, i32, ctypes.c_int64, i32]
    lib.tabi_arena_bytes.restype = ctypes.c_size_t
    for f in ("tabi_pack", "tabi_pack_device"):
        getattr(lib, f).argtypes = [P, P, i32, i32, i32, P, P, i32, P, P, P]
        getattr(lib, f).restype = ctypes.c_int
    lib.tabi_inspect.argtypes = [P, i32, i32, P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    lib.tabi_inspect.restype = ctypes.c_int
    lib.tabi_stage_times.argtypes = [P, i32, P, P, P]
    lib.tabi_stage_times.restype = ctypes.c_int
    _lib = lib
    return lib


def params_default(**kw) -> Params:
    p = Params()
    load().tabi_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def status_str(s: int) -> str:
    return load().tabi_status_str(int(s)).decode()


def sum_extent_texels(cs) -> int:
    """Sum over charts of input AABB width + height, whole texels (host-side
    sizing of the arena only)."""
    v = cs.verts.reshape(-1, 2).astype(np.int64)
    seg = np.repeat(np.arange(cs.n), np.diff(cs.offsets.astype(np.int64)))
    mn = np.full((cs.n, 2), np.iinfo(np.int64).max)
    mx = np.full((cs.n, 2), np.iinfo(np.int64).min)
    np.minimum.at(mn, seg, v)
    np.maximum.at(mx, seg, v)
    ext = (mx - mn + 255) // 256
    return int(ext.sum()) + 2 * cs.n


def arena_bytes(cs, gutter: int = 1) -> int:
    return int(load().tabi_arena_bytes(cs.n, cs.nv, cs.atlas_w, cs.atlas_h, sum_extent_texels(cs), gutter))


@dataclass
class PackResult:
    status: int
    k: int
    place: np.ndarray  # PLACEMENT_DTYPE[n], input order


class Context:
    """A packer context on one device with a torch-allocated arena."""

    def __init__(self, arena_bytes: int, device: int = 0):
        import torch
        self.lib = load()
        self.device = device
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=f"cuda:{device}")
        h = ctypes.c_void_p()
        st = self.lib.tabi_ctx_create(ctypes.byref(h), device, ctypes.c_void_p(self.arena.data_ptr()),
                                      ctypes.c_size_t(int(arena_bytes)))
        if st != TABI_OK:
            raise RuntimeError(f"tabi_ctx_create failed: {status_str(st)}")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.tabi_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return self.lib.tabi_last_error(self.h).decode()

    def pack(self, cs, params: Params | None = None, stream=None, out: np.ndarray | None = None) -> PackResult:
        """tabi_pack with host buffers (numpy; pinned if the caller made them so)."""
        params = params or params_default()
        offs = np.ascontiguousarray(cs.offsets, np.uint32)
        verts = np.ascontiguousarray(cs.verts, np.int32)
        if out is None:
            out = np.zeros(cs.n, PLACEMENT_DTYPE)
        k = ctypes.c_int32(0)
        st = self.lib.tabi_pack(self.h, ctypes.byref(params), cs.atlas_w, cs.atlas_h, cs.n,
                                offs.ctypes.data_as(ctypes.c_void_p), verts.ctypes.data_as(ctypes.c_void_p),
                                cs.nv, out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(k),
                                ctypes.c_void_p(_stream_ptr(stream)))
        return PackResult(int(st), int(k.value), out)

    def pack_host_ptrs(self, n, nv, W, H, offs_ptr, verts_ptr, out_ptr, params=None, stream=None):
        """tabi_pack on raw host pointers (e.g. pinned torch tensors)."""
        params = params or params_default()
        k = ctypes.c_int32(0)
        st = self.lib.tabi_pack(self.h, ctypes.byref(params), W, H, n, ctypes.c_void_p(offs_ptr),
                                ctypes.c_void_p(verts_ptr), nv, ctypes.c_void_p(out_ptr), ctypes.byref(k),
                                ctypes.c_void_p(_stream_ptr(stream)))
        return int(st), int(k.value)

    def pack_device(self, n, nv, W, H, offs_t, verts_t, out_t, params=None, stream=None):
        """tabi_pack_device: offs_t (int32/uint32 view), verts_t (int32) and
        out_t (uint8, 12*n bytes) are CUDA tensors."""
        params = params or params_default()
        k = ctypes.c_int32(0)
        st = self.lib.tabi_pack_device(self.h, ctypes.byref(params), W, H, n,
                                       ctypes.c_void_p(offs_t.data_ptr()), ctypes.c_void_p(verts_t.data_ptr()),
                                       nv, ctypes.c_void_p(out_t.data_ptr()), ctypes.byref(k),
                                       ctypes.c_void_p(_stream_ptr(stream)))
        return int(st), int(k.value)

    def stage_times(self, enable: bool):
        """Accumulated per-stage device ms and launch counts since the last
        call; then switches timing on or off (and clears the totals)."""
        ms = np.zeros(8, np.float64)
        launches = np.zeros(8, np.int64)
        packs = ctypes.c_int64(0)
        st = self.lib.tabi_stage_times(self.h, 1 if enable else 0, ms.ctypes.data_as(ctypes.c_void_p),
                                       launches.ctypes.data_as(ctypes.c_void_p), ctypes.byref(packs))
        if st != TABI_OK:
            raise RuntimeError(f"tabi_stage_times failed: {self.last_error()}")
        return dict(zip(STAGES, ms)), dict(zip(STAGES, launches)), int(packs.value)

    # ---- inspection of the last pack ------------------------------------
    def _inspect(self, what: int, scale: int = 0) -> bytes:
        need = ctypes.c_size_t(0)
        self.lib.tabi_inspect(self.h, what, scale, None, 0, ctypes.byref(need))
        buf = np.zeros(need.value, np.uint8)
        st = self.lib.tabi_inspect(self.h, what, scale, buf.ctypes.data_as(ctypes.c_void_p), need.value,
                                   ctypes.byref(need))
        if st != TABI_OK:
            raise RuntimeError(f"tabi_inspect failed: {self.last_error()}")
        return buf

    def charts(self) -> np.ndarray:
        return self._inspect(INSPECT_CHARTS).view(CHART_INFO_DTYPE)

    def perm(self) -> np.ndarray:
        return self._inspect(INSPECT_PERM).view(np.int32)

    def envelopes(self, scale: int, n: int):
        """List of (w', h', top', bot', left', right', maxbot) per sorted chart."""
        raw = self._inspect(INSPECT_ENV, scale)
        col_stride, row_stride = (int(v) for v in raw[:16].view(np.int64))
        meta = raw[16:16 + 16 * n].view(np.int32).reshape(n, 4)
        cols = raw[16 + 16 * n:16 + 16 * n + 4 * col_stride].view(np.uint32)
        rows = raw[16 + 16 * n + 4 * col_stride:].view(np.uint32)
        roff = self._inspect(INSPECT_ENV_CAP).view(np.int32).reshape(n, 2)[:, 0]
        out = []
        for s in range(n):
            wp, hp, cst, mb = (int(v) for v in meta[s])
            c = cols[cst:cst + wp]
            r = rows[roff[s]:roff[s] + hp]
            out.append((wp, hp, (c & 0xffff).astype(np.int32), (c >> 16).astype(np.int32),
                        (r & 0xffff).astype(np.int32), (r >> 16).astype(np.int32), mb))
        return out

    def pairs(self, scale: int, n: int):
        raw = self._inspect(INSPECT_PAIRS, scale)
        d = raw[:4 * n].view(np.int32)
        fl = raw[4 * n:4 * n + n]
        return d, (fl & 1).astype(np.uint8), ((fl >> 1) & 1).astype(np.uint8)

    def scale_result(self, scale: int, n: int):
        raw = self._inspect(INSPECT_SCALE, scale)
        hdr = raw[:32].view(np.int32)
        place = raw[32:32 + 16 * n].view(np.int32).reshape(n, 4)
        return hdr, place


def _stream_ptr(stream) -> int:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)
