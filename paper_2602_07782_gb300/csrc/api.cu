// C ABI of the packer (include/tabi.h): context, arena carving, the launch
// sequence of one pack, result selection and inspection.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>

#include "tabi_internal.cuh"

using namespace tabi;

struct tabi_ctx {
  int device = 0;
  char *arena = nullptr;
  size_t arena_bytes = 0;
  bool owned = false;
  std::atomic<int> busy{0};
  std::string last_error;
  Pack last{};  // device layout of the last pack, for tabi_inspect
  bool has_last = false;
  PackResult *host_result = nullptr;  // pinned
  // optional per-stage timing
  bool timing = false;
  cudaEvent_t ev[2 + 3 * 64 * 2 + 16] = {};
  int n_ev = 0;
  double stage_ms[8] = {};
  int64_t launches[8] = {};
  int64_t packs = 0;
};

namespace {

struct Guard {
  tabi_ctx *c;
  bool ok;
  explicit Guard(tabi_ctx *ctx) : c(ctx), ok(false) {
    int expect = 0;
    ok = c->busy.compare_exchange_strong(expect, 1);
  }
  ~Guard() {
    if (ok) c->busy.store(0);
  }
};

tabi_status fail(tabi_ctx *c, tabi_status s, const std::string &msg) {
  if (c) c->last_error = msg;
  return s;
}

tabi_status cuda_fail(tabi_ctx *c, cudaError_t e, const char *where) {
  return fail(c, TABI_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// bump allocator over the arena (256-byte aligned pieces)
struct Carve {
  char *base;
  size_t cap, used = 0;
  template <typename T>
  T *take(size_t count) {
    const size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
    if (used + bytes > cap) return nullptr;
    T *p = reinterpret_cast<T *>(base + used);
    used += bytes;
    return p;
  }
};

bool valid_params(const tabi_params *p) {
  return p && p->version == TABI_PARAMS_VERSION && p->gutter >= 0 && p->gutter <= kMaxGutter &&
         p->knee_abs_pct >= 0 && p->knee_abs_pct <= 100 && p->knee_rel_pct >= 0 &&
         p->knee_rel_pct <= 100 && p->lr_sig_pct >= 0 && p->lr_sig_pct <= 100 &&
         p->knee_margin >= 0 && p->knee_margin <= 1 << 20 && (p->flags & ~TABI_F_ALL) == 0 &&
         p->scale_fanout >= 1 && p->scale_fanout <= kScales;
}

size_t fixed_bytes(int64_t n, int64_t nv) {
  size_t b = 0;
  auto add = [&](size_t x) { b += (x + 255) & ~(size_t)255; };
  add(4 * (n + 1));              // offsets (host variant)
  add(8 * nv);                   // verts (host variant)
  add(sizeof(tabi_chart_info) * n);
  add(sizeof(ChartShape) * n * 2);
  add(4 * n);                    // perm
  add(4 * n);                    // hq
  add(16 * n);                   // sort ping-pong
  add(8 * n);                    // env_off
  add((size_t)kScales * 4 * n);  // colstart
  add((size_t)kScales * 16 * n); // meta
  add((size_t)kScales * 4 * n);  // dnext
  add((size_t)kScales * n);      // pflags
  add((size_t)kScales * 16 * n); // place
  add(sizeof(ScaleOut) * kScales);
  add(4);                        // found
  add(sizeof(PackResult));
  add(4);                        // err
  add(sizeof(tabi_placement) * n);
  return b + 4096;
}

__global__ void init_kernel(Pack p) {
  const int t = threadIdx.x;
  if (t < kScales) p.scale_out[t] = ScaleOut{0, 0, 0, 0, 0, 0, 0, 0};
  if (t == 0) {
    *p.found = -1;
    *p.err = 0;
    *p.result = PackResult{0, 0, 0, -1};
  }
}

// Largest successful candidate (Sec. 3.1 / Sec. 5), then the placements of
// that candidate gathered back into input order.
__global__ void select_kernel(Pack p) {
  __shared__ int best;
  __shared__ uint32_t err;
  if (threadIdx.x == 0) {
    int b = -1;
    for (int j = kScales - 1; j >= 0; --j)
      if (p.scale_out[j].success) { b = j; break; }
    best = b;
    err = *p.err;
    PackResult r{0, 0, err, b};
    if (err & kErrInvalid) r.status = TABI_ERR_INVALID_ARG;
    else if (err & (kErrPool | kErrRow)) r.status = TABI_ERR_OOM;
    else if (b < 0) r.status = TABI_ERR_NO_FIT;
    else { r.status = TABI_OK; r.k = 16 * (b + 1); }
    *p.result = r;
  }
  __syncthreads();
  if (best < 0 || err) return;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < p.n; s += gridDim.x * blockDim.x) {
    const int c = p.perm[s];
    const int4 pl = p.place[(int64_t)best * p.n + s];
    const tabi_chart_info &inf = p.info[c];
    tabi_placement o;
    o.x = pl.x;
    o.y = pl.y;
    o.rot90 = (uint8_t)inf.rot90;
    o.flip_x = (uint8_t)inf.flip_x;
    o.flip_y = (uint8_t)inf.flip_y;
    o.mirror = (uint8_t)(pl.w & 1);
    p.out[c] = o;
  }
}

// Event pairs around each stage of one pack: (stage, start event, end event)
struct StageMarks {
  tabi_ctx *c;
  cudaStream_t st;
  int used = 0;
  int stage[128];
  void mark_begin(int s) {
    if (!c->timing || used >= 128) return;
    stage[used] = s;
    cudaEventRecord(c->ev[2 * used], st);
  }
  void mark_end() {
    if (!c->timing || used >= 128) return;
    cudaEventRecord(c->ev[2 * used + 1], st);
    ++used;
  }
  void collect() {
    if (!c->timing) return;
    float total = 0.f;
    for (int i = 0; i < used; ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]);
      c->stage_ms[stage[i]] += ms;
      c->launches[stage[i]] += 1;
    }
    if (used) cudaEventElapsedTime(&total, c->ev[0], c->ev[2 * used - 1]);
    c->stage_ms[7] += total;
    c->launches[7] += 1;
    c->packs += 1;
  }
};

tabi_status run_pack(tabi_ctx *ctx, const tabi_params *params, int32_t W, int32_t H, int32_t n,
                     const uint32_t *offsets, const int32_t *verts, int32_t nv, tabi_placement *out,
                     int32_t *out_k, void *stream, bool host) {
  if (!ctx) return TABI_ERR_INVALID_ARG;
  Guard g(ctx);
  if (!g.ok) return fail(ctx, TABI_ERR_BUSY, "context in use");
  if (!valid_params(params)) return fail(ctx, TABI_ERR_INVALID_ARG, "bad params");
  if (n < 1 || nv < 3 || W < 1 || H < 1 || W > kMaxAtlas || H > kMaxAtlas || !offsets || !verts ||
      !out || !out_k)
    return fail(ctx, TABI_ERR_INVALID_ARG, "bad sizes or null pointer");
  if (host) {
    if (offsets[0] != 0 || offsets[n] != (uint32_t)nv)
      return fail(ctx, TABI_ERR_INVALID_ARG, "offsets must run from 0 to n_verts");
  }
  *out_k = 0;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  if (rowloop_smem_bytes(W, params->gutter) > (size_t)smem_optin)
    return fail(ctx, TABI_ERR_INVALID_ARG, "atlas too wide for this gutter: the row working set exceeds shared memory");

  Carve cv{ctx->arena, ctx->arena_bytes};
  Pack p{};
  p.n = n; p.nv = nv; p.W = W; p.H = H; p.g = params->gutter;
  p.knee_abs = params->knee_abs_pct; p.knee_rel = params->knee_rel_pct;
  p.lr_sig = params->lr_sig_pct; p.knee_margin = params->knee_margin;
  p.flags = params->flags;
  uint32_t *d_off = nullptr;
  int32_t *d_verts = nullptr;
  if (host) {
    d_off = cv.take<uint32_t>(n + 1);
    d_verts = cv.take<int32_t>(2 * (size_t)nv);
  }
  p.info = cv.take<tabi_chart_info>(n);
  p.shape_in = cv.take<ChartShape>(n);
  p.shape = cv.take<ChartShape>(n);
  p.perm = cv.take<int32_t>(n);
  p.hq = cv.take<int32_t>(n);
  p.sort_tmp = cv.take<uint32_t>(4 * (size_t)n);
  p.env_off = cv.take<int32_t>(2 * (size_t)n);
  p.colstart = cv.take<int32_t>((size_t)kScales * n);
  p.meta = cv.take<int32_t>((size_t)kScales * 4 * n);
  p.dnext = cv.take<int32_t>((size_t)kScales * n);
  p.pflags = cv.take<uint8_t>((size_t)kScales * n);
  p.place = cv.take<int4>((size_t)kScales * n);
  p.scale_out = cv.take<ScaleOut>(kScales);
  p.found = cv.take<int32_t>(1);
  p.result = cv.take<PackResult>(1);
  p.err = cv.take<uint32_t>(1);
  tabi_placement *d_out = host ? cv.take<tabi_placement>(n) : out;
  if (!p.info || !p.shape || !p.place || !p.err || !p.colstart || !d_out || (host && (!d_off || !d_verts)))
    return fail(ctx, TABI_ERR_OOM, "arena too small for the per-chart arrays");
  const size_t left = (cv.cap - cv.used) / sizeof(uint32_t);
  // the rest in equal thirds: column words, their chart indices, row words
  p.col_stride = p.row_stride = (int64_t)(left / (3 * kScales)) & ~(int64_t)63;
  p.colpool = reinterpret_cast<uint32_t *>(cv.base + cv.used);
  p.colown = reinterpret_cast<int32_t *>(p.colpool + (int64_t)kScales * p.col_stride);
  p.pool = reinterpret_cast<uint32_t *>(p.colown + (int64_t)kScales * p.col_stride);
  if (p.col_stride < 64) return fail(ctx, TABI_ERR_OOM, "arena too small for the envelope pools");
  p.offsets = host ? d_off : offsets;
  p.verts = host ? d_verts : verts;
  p.out = d_out;

  if (host) {
    e = cudaMemcpyAsync(d_off, offsets, sizeof(uint32_t) * (n + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_verts, verts, sizeof(int32_t) * 2 * (size_t)nv, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "input copy");
  }
  StageMarks mk{ctx, st};
  mk.mark_begin(0);
  init_kernel<<<1, 64, 0, st>>>(p);
  launch_prep(p, st);
  mk.mark_end();
  mk.mark_begin(1);
  launch_sort(p, st);
  mk.mark_end();
  mk.mark_begin(2);
  launch_layout(p, st);
  mk.mark_end();
  // descending search in waves of `scale_fanout` candidates; once a wave
  // has a success every later kernel returns at entry
  const int F = params->scale_fanout;
  for (int j_hi = kScales - 1; j_hi >= 0; j_hi -= F) {
    const int j_lo = j_hi - F + 1 < 0 ? 0 : j_hi - F + 1;
    mk.mark_begin(3);
    launch_raster(p, j_lo, j_hi, st);
    mk.mark_end();
    mk.mark_begin(4);
    launch_hcompact(p, j_lo, j_hi, st);
    mk.mark_end();
    mk.mark_begin(5);
    e = launch_rowloop(p, j_lo, j_hi, st);
    mk.mark_end();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "rowloop launch");
  }
  mk.mark_begin(6);
  select_kernel<<<(n + 255) / 256 < 148 ? (n + 255) / 256 : 148, 256, 0, st>>>(p);
  mk.mark_end();
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");
  e = cudaMemcpyAsync(ctx->host_result, p.result, sizeof(PackResult), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && host)
    e = cudaMemcpyAsync(out, d_out, sizeof(tabi_placement) * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pack");
  mk.collect();
  ctx->last = p;
  ctx->has_last = true;
  const PackResult r = *ctx->host_result;
  if (r.status == TABI_OK) *out_k = r.k;
  switch (r.status) {
    case TABI_OK: return TABI_OK;
    case TABI_ERR_NO_FIT: return fail(ctx, TABI_ERR_NO_FIT, "no candidate scale fits every chart");
    case TABI_ERR_INVALID_ARG: return fail(ctx, TABI_ERR_INVALID_ARG, "invalid chart (vertices, size or range)");
    default: return fail(ctx, TABI_ERR_OOM, "arena too small for the envelopes of this input");
  }
}

}  // namespace

extern "C" {

void tabi_params_default(tabi_params *p) {
  if (!p) return;
  p->version = TABI_PARAMS_VERSION;
  p->gutter = 1;
  p->knee_abs_pct = 10;
  p->knee_rel_pct = 20;
  p->lr_sig_pct = 10;
  p->knee_margin = 1;
  p->flags = TABI_F_ALL;
  p->scale_fanout = kScales;
}

tabi_status tabi_ctx_create(tabi_ctx **out, int device, void *arena, size_t arena_bytes) {
  if (!out) return TABI_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return TABI_ERR_INVALID_ARG;
  if (arena && ((uintptr_t)arena & 255)) return TABI_ERR_INVALID_ARG;
  if (arena_bytes < (1u << 20)) return TABI_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return TABI_ERR_CUDA;
  tabi_ctx *c = new tabi_ctx();
  c->device = device;
  c->arena_bytes = arena_bytes;
  if (arena) {
    c->arena = (char *)arena;
  } else {
    if (cudaMalloc(&c->arena, arena_bytes) != cudaSuccess) { delete c; return TABI_ERR_CUDA; }
    c->owned = true;
  }
  if (cudaMallocHost(&c->host_result, sizeof(PackResult)) != cudaSuccess) {
    if (c->owned) cudaFree(c->arena);
    delete c;
    return TABI_ERR_CUDA;
  }
  *out = c;
  return TABI_OK;
}

void tabi_ctx_destroy(tabi_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  for (int i = 0; i < c->n_ev; ++i) cudaEventDestroy(c->ev[i]);
  if (c->owned) cudaFree(c->arena);
  if (c->host_result) cudaFreeHost(c->host_result);
  delete c;
}

const char *tabi_last_error(const tabi_ctx *c) { return c ? c->last_error.c_str() : "null context"; }

const char *tabi_status_str(tabi_status s) {
  switch (s) {
    case TABI_OK: return "ok";
    case TABI_ERR_INVALID_ARG: return "invalid argument";
    case TABI_ERR_NO_FIT: return "no candidate scale fits";
    case TABI_ERR_OOM: return "arena too small";
    case TABI_ERR_CUDA: return "CUDA error";
    case TABI_ERR_TIMEOUT: return "timeout";
    case TABI_ERR_BUSY: return "context busy";
  }
  return "unknown status";
}

size_t tabi_arena_bytes(int32_t n, int32_t nv, int32_t W, int32_t H, int64_t sum_extent_texels,
                        int32_t gutter) {
  (void)W; (void)H;
  if (n < 1) return 0;
  // column words, their chart indices and row words get equal shares; each
  // must hold the larger of sum(w') and sum(h') at k = 1024, both below
  // sum_extent + n (2g + 4)
  const size_t pool = (size_t)kScales * 4 * 3 *
                      ((size_t)sum_extent_texels + (size_t)n * (2 * (size_t)gutter + 4) + 64);
  return fixed_bytes(n, nv) + pool + (size_t)kScales * 256;
}

tabi_status tabi_pack(tabi_ctx *ctx, const tabi_params *params, int32_t W, int32_t H, int32_t n,
                      const uint32_t *offsets, const int32_t *verts, int32_t nv, tabi_placement *out,
                      int32_t *out_k, void *stream) {
  return run_pack(ctx, params, W, H, n, offsets, verts, nv, out, out_k, stream, true);
}

tabi_status tabi_pack_device(tabi_ctx *ctx, const tabi_params *params, int32_t W, int32_t H,
                             int32_t n, const uint32_t *offsets, const int32_t *verts, int32_t nv,
                             tabi_placement *out, int32_t *out_k, void *stream) {
  return run_pack(ctx, params, W, H, n, offsets, verts, nv, out, out_k, stream, false);
}

tabi_status tabi_stage_times(tabi_ctx *ctx, int32_t enable, double *stage_ms, int64_t *launches,
                             int64_t *packs) {
  if (!ctx) return TABI_ERR_INVALID_ARG;
  Guard g(ctx);
  if (!g.ok) return fail(ctx, TABI_ERR_BUSY, "context in use");
  if (stage_ms) for (int i = 0; i < 8; ++i) stage_ms[i] = ctx->stage_ms[i];
  if (launches) for (int i = 0; i < 8; ++i) launches[i] = ctx->launches[i];
  if (packs) *packs = ctx->packs;
  if (enable && ctx->n_ev == 0) {
    cudaSetDevice(ctx->device);
    const int want = (int)(sizeof(ctx->ev) / sizeof(ctx->ev[0]));
    for (int i = 0; i < want; ++i) {
      const cudaError_t e = cudaEventCreate(&ctx->ev[i]);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventCreate");
      ctx->n_ev = i + 1;
    }
  }
  for (int i = 0; i < 8; ++i) { ctx->stage_ms[i] = 0; ctx->launches[i] = 0; }
  ctx->packs = 0;
  ctx->timing = enable != 0;
  return TABI_OK;
}

tabi_status tabi_inspect(tabi_ctx *ctx, int32_t what, int32_t scale, void *dst, size_t cap,
                         size_t *needed) {
  if (!ctx || !ctx->has_last || !needed) return TABI_ERR_INVALID_ARG;
  Guard g(ctx);
  if (!g.ok) return fail(ctx, TABI_ERR_BUSY, "context in use");
  const Pack &p = ctx->last;
  const size_t n = (size_t)p.n;
  if (scale < 0 || scale >= kScales) return fail(ctx, TABI_ERR_INVALID_ARG, "bad scale index");
  struct Piece { const void *src; size_t bytes; bool host; };
  const int64_t strides[2] = {p.col_stride, p.row_stride};
  Piece pcs[4] = {{nullptr, 0, false}, {nullptr, 0, false}, {nullptr, 0, false}, {nullptr, 0, false}};
  switch (what) {
    case TABI_INSPECT_CHARTS: pcs[0] = {p.info, sizeof(tabi_chart_info) * n, false}; break;
    case TABI_INSPECT_PERM: pcs[0] = {p.perm, 4 * n, false}; break;
    case TABI_INSPECT_ENV:
      pcs[0] = {strides, sizeof(strides), true};
      pcs[1] = {p.meta + (int64_t)scale * 4 * n, 16 * n, false};
      pcs[2] = {p.colpool + (int64_t)scale * p.col_stride, 4 * (size_t)p.col_stride, false};
      pcs[3] = {p.pool + (int64_t)scale * p.row_stride, 4 * (size_t)p.row_stride, false};
      break;
    case TABI_INSPECT_ENV_CAP: pcs[0] = {p.env_off, 8 * n, false}; break;
    case TABI_INSPECT_PAIRS:
      pcs[0] = {p.dnext + (int64_t)scale * n, 4 * n, false};
      pcs[1] = {p.pflags + (int64_t)scale * n, (size_t)n, false};
      break;
    case TABI_INSPECT_SCALE:
      pcs[0] = {p.scale_out + scale, sizeof(ScaleOut), false};
      pcs[1] = {p.place + (int64_t)scale * n, 16 * n, false};
      break;
    default: return fail(ctx, TABI_ERR_INVALID_ARG, "bad inspect selector");
  }
  *needed = pcs[0].bytes + pcs[1].bytes + pcs[2].bytes + pcs[3].bytes;
  if (!dst || cap < *needed) return fail(ctx, TABI_ERR_INVALID_ARG, "buffer too small");
  cudaSetDevice(ctx->device);
  char *d = (char *)dst;
  for (const Piece &pc : pcs) {
    if (!pc.bytes) continue;
    if (pc.host) {
      memcpy(d, pc.src, pc.bytes);
    } else {
      const cudaError_t e = cudaMemcpy(d, pc.src, pc.bytes, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "inspect copy");
    }
    d += pc.bytes;
  }
  return TABI_OK;
}

}  // extern "C"
