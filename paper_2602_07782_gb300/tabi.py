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

(TABI_OK, TABI_ERR_INVALID_ARG, TABI_ERR_NO_FIT, TABI_ERR_OOM, TABI_ERR_CUDA, TABI_ERR_TIMEOUT, TABI_ERR_BUSY,
 TABI_PENDING) = range(8)
F_HC, F_BALANCE, F_OBB, F_LAABB = 1, 2, 4, 8
F_ALL = 15
F_EVAL_ALL = 16  # inspection aid: every candidate's row loop runs to its end
INSPECT_CHARTS, INSPECT_PERM, INSPECT_ENV, INSPECT_REGIONS, INSPECT_PAIRS, INSPECT_SCALE = 1, 2, 3, 4, 5, 6
N_SCALES = 64
MAX_CHARTS = 131072
MAX_BATCH = 65536


class Params(ctypes.Structure):
    _fields_ = [("version", ctypes.c_int32), ("gutter", ctypes.c_int32),
                ("knee_abs_pct", ctypes.c_int32), ("knee_rel_pct", ctypes.c_int32),
                ("lr_sig_pct", ctypes.c_int32), ("knee_margin", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("scale_fanout", ctypes.c_int32),
                ("laabb_count", ctypes.c_int32), ("topt_permille", ctypes.c_int32),
                ("hybrid_min_charts", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("atlas_w", ctypes.c_int32), ("atlas_h", ctypes.c_int32),
                ("n_charts", ctypes.c_int32), ("n_verts", ctypes.c_int32),
                ("offsets", ctypes.c_void_p), ("verts", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("scale_k", ctypes.c_int32), ("status", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("scale_fanout", ctypes.c_int32), ("raster_warp_items", ctypes.c_int32),
                ("rowloop_threads", ctypes.c_int32), ("rowloop_ctas", ctypes.c_int32), ("chunks", ctypes.c_int32),
                ("progressive_bound", ctypes.c_int32), ("ms", ctypes.c_float)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("lanes", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("check", ctypes.c_int32), ("arena_bytes", ctypes.c_size_t), ("params", Params)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("scale_k", ctypes.c_int32), ("t_submit_ns", ctypes.c_int64),
                ("t_start_ns", ctypes.c_int64), ("t_done_ns", ctypes.c_int64),
                ("overlap_texels", ctypes.c_int64), ("gutter_texels", ctypes.c_int64),
                ("outside_texels", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("submitted", "launched", "completed", "batches", "max_batch",
                                              "queued", "busy_lanes", "checked", "check_violations",
                                              "check_ns")]


class Quality(ctypes.Structure):
    _fields_ = [("overlap_texels", ctypes.c_int64), ("gutter_texels", ctypes.c_int64),
                ("outside_texels", ctypes.c_int64)]


PLACEMENT_DTYPE = np.dtype([("x", "<i4"), ("y", "<i4"), ("rot90", "u1"), ("flip_x", "u1"),
                            ("flip_y", "u1"), ("mirror", "u1"), ("k", "<i4")])

CHART_INFO_DTYPE = np.dtype([
    ("orig", "<i4"), ("Wq", "<i4"), ("Hq", "<i4"), ("rot90", "<i4"), ("flip_y", "<i4"),
    ("flip_x", "<i4"), ("obb_m", "<i4"), ("valid", "<i4"),
    ("u0", "<i8"), ("u1", "<i8"), ("v0", "<i8"), ("v1", "<i8"),
    ("ylo", "<i4", 10), ("yhi", "<i4", 10), ("xlo", "<i4", 10), ("xhi", "<i4", 10),
    ("area_top", "<i8"), ("area_bot", "<i8"), ("area_left", "<i8"), ("area_right", "<i8"),
    ("area_bl2", "<i8"), ("area_br2", "<i8")])

EXPORTS = ["tabi_params_default", "tabi_ctx_create", "tabi_ctx_destroy", "tabi_last_error",
           "tabi_status_str", "tabi_arena_bytes", "tabi_pack", "tabi_pack_device", "tabi_pack_batch",
           "tabi_pack_batch_device", "tabi_pack_batch_shaped", "tabi_autotune", "tabi_inspect", "tabi_inspect_atlas",
           "tabi_stage_times", "tabi_server_config_default", "tabi_server_create", "tabi_server_destroy",
           "tabi_submit", "tabi_poll", "tabi_wait", "tabi_server_get_stats", "tabi_check_packing_device",
           "tabi_sort_heights_noalloc", "tabi_measure_int_rate"]
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
    for f in ("tabi_pack_batch", "tabi_pack_batch_device"):
        getattr(lib, f).argtypes = [P, P, P, i32, P]
        getattr(lib, f).restype = ctypes.c_int
    lib.tabi_autotune.argtypes = [P, P, P, i32, P, P]
    lib.tabi_autotune.restype = ctypes.c_int
    lib.tabi_pack_batch_shaped.argtypes = [P, P, P, i32, P, i32, P]
    lib.tabi_pack_batch_shaped.restype = ctypes.c_int
    lib.tabi_server_config_default.argtypes = [P]
    lib.tabi_server_create.argtypes = [ctypes.POINTER(P), P]
    lib.tabi_server_create.restype = ctypes.c_int
    lib.tabi_server_destroy.argtypes = [P]
    lib.tabi_submit.argtypes = [P, P, ctypes.POINTER(ctypes.c_uint64)]
    lib.tabi_submit.restype = ctypes.c_int
    lib.tabi_poll.argtypes = [P, ctypes.c_uint64, P]
    lib.tabi_poll.restype = ctypes.c_int
    lib.tabi_wait.argtypes = [P, ctypes.c_uint64, i32, P]
    lib.tabi_wait.restype = ctypes.c_int
    lib.tabi_server_get_stats.argtypes = [P, P]
    lib.tabi_server_get_stats.restype = ctypes.c_int
    lib.tabi_inspect.argtypes = [P, i32, i32, P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    lib.tabi_inspect.restype = ctypes.c_int
    lib.tabi_inspect_atlas.argtypes = [P, i32, i32, i32, P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    lib.tabi_inspect_atlas.restype = ctypes.c_int
    lib.tabi_stage_times.argtypes = [P, i32, P, P, P]
    lib.tabi_stage_times.restype = ctypes.c_int
    lib.tabi_check_packing_device.argtypes = [P, i32, i32, i32, i32, P, P, i32, P, P, P]
    lib.tabi_check_packing_device.restype = ctypes.c_int
    lib.tabi_measure_int_rate.argtypes = [i32, ctypes.POINTER(ctypes.c_double)]
    lib.tabi_measure_int_rate.restype = ctypes.c_int
    _lib = lib
    return lib


def params_default(**kw) -> Params:
    p = Params()
    load().tabi_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def measure_int_rate(device: int = 0) -> float:
    """tabi_measure_int_rate: the device's integer-operation rate of the
    rasterizer's mix, operations per second."""
    v = ctypes.c_double(0.0)
    st = load().tabi_measure_int_rate(device, ctypes.byref(v))
    if st != TABI_OK:
        raise RuntimeError(f"tabi_measure_int_rate failed: {status_str(st)}")
    return float(v.value)


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


def waves(fanout: int) -> int:
    """Waves of the descending scale search for a fan-out."""
    return (N_SCALES + fanout - 1) // fanout


def kernels_per_pack(fanout: int, chunks: int = 4, waves_run: int | None = None, tail: bool = False) -> int:
    """Kernels one (batched) pack launches: init, prep, sort + gather,
    layout + bases; per wave, for each chart chunk plan + fill, raster,
    compaction, row loop, then (if some atlas may take the prefix-sum tail)
    per tail round the tail's plan, four phases of trial offsets, trial
    scales and pick, redraw, compaction and push pass, then the wave's end;
    selection.  The graph runs waves only
    while some atlas still searches (`waves_run` of them: the most any
    atlas of the batch needs, at least one); direct launches (stage timing)
    run every wave."""
    w = waves(fanout) if waves_run is None else max(1, waves_run)
    return 7 + (5 * chunks + 1 + (16 * tail_rounds(fanout) if tail else 0)) * w


def tail_rounds(fanout: int) -> int:
    """Tail rounds per wave: quotas 1, 2, 4, ... tasks per atlas, the last
    round the rest (at most 7)."""
    r = 1
    while (1 << r) - 1 < fanout and r < 7:
        r += 1
    return r


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
        out_t (uint8, PLACEMENT_DTYPE.itemsize * n bytes) are CUDA tensors."""
        params = params or params_default()
        k = ctypes.c_int32(0)
        st = self.lib.tabi_pack_device(self.h, ctypes.byref(params), W, H, n,
                                       ctypes.c_void_p(offs_t.data_ptr()), ctypes.c_void_p(verts_t.data_ptr()),
                                       nv, ctypes.c_void_p(out_t.data_ptr()), ctypes.byref(k),
                                       ctypes.c_void_p(_stream_ptr(stream)))
        return int(st), int(k.value)

    def check_packing_device(self, W, H, gutter, n, nv, offs_t, verts_t, place_t, stream=None):
        """tabi_check_packing_device on CUDA tensors (offsets, vertices,
        placements as a uint8 view): the paper's overlap metric as
        (overlap, gutter, outside) texel counts."""
        q = Quality()
        st = self.lib.tabi_check_packing_device(self.h, W, H, gutter, n, ctypes.c_void_p(offs_t.data_ptr()),
                                                ctypes.c_void_p(verts_t.data_ptr()), nv,
                                                ctypes.c_void_p(place_t.data_ptr()), ctypes.byref(q),
                                                ctypes.c_void_p(_stream_ptr(stream)))
        return int(st), (int(q.overlap_texels), int(q.gutter_texels), int(q.outside_texels))

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

    def pack_batch(self, sets, params: Params | None = None, stream=None, outs=None, shape: Tuning | None = None):
        """tabi_pack_batch with host buffers: one ChartSet per atlas (with an
        explicit launch shape: tabi_pack_batch_shaped).  Returns (call status,
        [PackResult per atlas])."""
        params = params or params_default()
        keep = []
        reqs = (Request * len(sets))()
        outs = outs or [np.zeros(cs.n, PLACEMENT_DTYPE) for cs in sets]
        for i, cs in enumerate(sets):
            offs = np.ascontiguousarray(cs.offsets, np.uint32)
            verts = np.ascontiguousarray(cs.verts, np.int32)
            keep += [offs, verts]
            reqs[i] = Request(cs.atlas_w, cs.atlas_h, cs.n, cs.nv, offs.ctypes.data, verts.ctypes.data,
                              outs[i].ctypes.data, 0, 0)
        if shape is None:
            st = self.lib.tabi_pack_batch(self.h, ctypes.byref(params), reqs, len(sets),
                                          ctypes.c_void_p(_stream_ptr(stream)))
        else:
            st = self.lib.tabi_pack_batch_shaped(self.h, ctypes.byref(params), reqs, len(sets),
                                                 ctypes.c_void_p(_stream_ptr(stream)), 0, ctypes.byref(shape))
        return int(st), [PackResult(int(r.status), int(r.scale_k), o) for r, o in zip(reqs, outs)]

    def pack_batch_requests(self, reqs, params: Params | None = None, stream=None, device: bool = True):
        """tabi_pack_batch(_device) on a prepared ctypes Request array (raw
        pointers, e.g. into CUDA or pinned torch tensors); statuses and k are
        written into reqs."""
        params = params or params_default()
        f = self.lib.tabi_pack_batch_device if device else self.lib.tabi_pack_batch
        return int(f(self.h, ctypes.byref(params), reqs, len(reqs), ctypes.c_void_p(_stream_ptr(stream))))

    def autotune(self, reqs, params: Params | None = None, stream=None):
        """tabi_autotune on a prepared ctypes Request array (device pointers).
        Returns (status, Tuning)."""
        params = params or params_default()
        t = Tuning()
        st = self.lib.tabi_autotune(self.h, ctypes.byref(params), reqs, len(reqs),
                                    ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(t))
        return int(st), t

    # ---- inspection of the last pack ------------------------------------
    def _inspect(self, what: int, scale: int = 0, atlas: int = 0) -> np.ndarray:
        need = ctypes.c_size_t(0)
        self.lib.tabi_inspect_atlas(self.h, atlas, what, scale, None, 0, ctypes.byref(need))
        buf = np.zeros(need.value, np.uint8)
        st = self.lib.tabi_inspect_atlas(self.h, atlas, what, scale, buf.ctypes.data_as(ctypes.c_void_p),
                                         need.value, ctypes.byref(need))
        if st != TABI_OK:
            raise RuntimeError(f"tabi_inspect failed: {self.last_error()}")
        return buf

    def charts(self, atlas: int = 0) -> np.ndarray:
        return self._inspect(INSPECT_CHARTS, 0, atlas).view(CHART_INFO_DTYPE)

    def perm(self, atlas: int = 0) -> np.ndarray:
        return self._inspect(INSPECT_PERM, 0, atlas).view(np.int32)

    def envelopes(self, scale: int, n: int, atlas: int = 0):
        """List of (w', h', top', bot', left', right', maxbot) per sorted chart."""
        raw = self._inspect(INSPECT_ENV, scale, atlas)
        cwords, rwords = (int(v) for v in raw[:16].view(np.int64))
        o = 16
        meta = raw[o:o + 16 * n].view(np.int32).reshape(n, 4)
        o += 16 * n
        rst = raw[o:o + 4 * n].view(np.int32)
        o += 4 * n
        cols = raw[o:o + 4 * cwords].view(np.uint32)
        rows = raw[o + 4 * cwords:o + 4 * cwords + 4 * rwords].view(np.uint32)
        out = []
        for s in range(n):
            wp, hp, cst, mb = (int(v) for v in meta[s])
            c = cols[cst:cst + wp]
            r = rows[rst[s]:rst[s] + hp]
            out.append((wp, hp, (c & 0xffff).astype(np.int32), (c >> 16).astype(np.int32),
                        (r & 0xffff).astype(np.int32), (r >> 16).astype(np.int32), mb))
        return out

    def regions(self, atlas: int = 0):
        """(start[64, 2], words[64, 2], top candidate) of the atlas's column /
        row regions."""
        raw = self._inspect(INSPECT_REGIONS, 0, atlas).view(np.int64)
        return raw[:128].reshape(64, 2), raw[128:256].reshape(64, 2), int(raw[256])

    def waves_run(self) -> int:
        """Waves of candidates the last pack ran (its device-side loop stops
        once no atlas of the batch searches)."""
        return int(self._inspect(INSPECT_REGIONS, 0, 0).view(np.int64)[257])

    def prep_group(self) -> int:
        """Lanes per chart the last pack's prep used (32, 16, 8 or 4: wider
        while its charts leave the GPU's resident warps idle)."""
        return int(self._inspect(INSPECT_REGIONS, 0, 0).view(np.int64)[258])

    def raster_words(self) -> int:
        """Padded scanline words (columns + rows, every chart and candidate)
        the last pack's raster evaluated."""
        return int(self._inspect(INSPECT_REGIONS, 0, 0).view(np.int64)[259])

    def raster_column_words(self) -> int:
        """Padded column words among them (the rest are row words)."""
        return int(self._inspect(INSPECT_REGIONS, 0, 0).view(np.int64)[260])

    def pairs(self, scale: int, n: int, atlas: int = 0):
        raw = self._inspect(INSPECT_PAIRS, scale, atlas)
        d = raw[:4 * n].view(np.int32)
        fl = raw[4 * n:4 * n + n]
        return d, (fl & 1).astype(np.uint8), ((fl >> 1) & 1).astype(np.uint8)

    def scale_result(self, scale: int, n: int, atlas: int = 0):
        """(header int32[12], place int32[n, 4]) of candidate `scale`: success,
        rows, knee rows, knees, max frontline, placed, evaluated, tail rows,
        tail scale, first tail chart, then the area-weighted scale sum as
        header[12] (a Python int)."""
        raw = self._inspect(INSPECT_SCALE, scale, atlas)
        hdr = raw[:48].view(np.int32).copy()
        lo, hi = (int(v) for v in raw[48:64].view(np.uint64))
        place = raw[64:64 + 16 * n].view(np.int32).reshape(n, 4)
        return [int(v) for v in hdr] + [(hi << 64) | lo], place


def server_config_default(**kw) -> ServerConfig:
    c = ServerConfig()
    load().tabi_server_config_default(ctypes.byref(c))
    for k, v in kw.items():
        if k == "params":
            c.params = v
        else:
            setattr(c, k, v)
    return c


class Server:
    """Serving loop (continuous batching) on one device: tabi_server_*."""

    def __init__(self, cfg: ServerConfig | None = None, **kw):
        self.lib = load()
        cfg = cfg or server_config_default(**kw)
        h = ctypes.c_void_p()
        st = self.lib.tabi_server_create(ctypes.byref(h), ctypes.byref(cfg))
        if st != TABI_OK:
            raise RuntimeError(f"tabi_server_create failed: {status_str(st)}")
        self.h = h
        self._held = {}  # ticket -> buffers that must outlive the request

    def submit(self, cs, out: np.ndarray | None = None):
        """Queue one ChartSet (host buffers).  Returns (status, ticket, out)."""
        offs = np.ascontiguousarray(cs.offsets, np.uint32)
        verts = np.ascontiguousarray(cs.verts, np.int32)
        if out is None:
            out = np.zeros(cs.n, PLACEMENT_DTYPE)
        return self.submit_ptrs(cs.n, cs.nv, cs.atlas_w, cs.atlas_h, offs, verts, out)

    def submit_ptrs(self, n, nv, W, H, offs: np.ndarray, verts: np.ndarray, out: np.ndarray):
        req = Request(W, H, n, nv, offs.ctypes.data, verts.ctypes.data, out.ctypes.data, 0, 0)
        t = ctypes.c_uint64(0)
        st = self.lib.tabi_submit(self.h, ctypes.byref(req), ctypes.byref(t))
        if st == TABI_OK:
            self._held[int(t.value)] = (offs, verts, out)
        return int(st), int(t.value), out

    def _done(self, ticket, st, r):
        if st == TABI_OK:
            self._held.pop(ticket, None)
        return st, r

    def poll(self, ticket: int):
        r = Result()
        st = self.lib.tabi_poll(self.h, ticket, ctypes.byref(r))
        return self._done(ticket, int(st), r)

    def wait(self, ticket: int, timeout_ms: int = 60000):
        r = Result()
        st = self.lib.tabi_wait(self.h, ticket, int(timeout_ms), ctypes.byref(r))
        return self._done(ticket, int(st), r)

    def stats(self) -> dict:
        s = ServerStats()
        self.lib.tabi_server_get_stats(self.h, ctypes.byref(s))
        return {f: int(getattr(s, f)) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.lib.tabi_server_destroy(self.h)
            self.h = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


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
