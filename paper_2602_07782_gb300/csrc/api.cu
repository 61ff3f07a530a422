// C ABI of the packer (include/tabi.h): context, arena carving, the launch
// sequence of a batch of atlases (captured once per wave structure into a
// CUDA graph and replayed), per-atlas results and inspection.  A single
// pack is a batch of one.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "context.h"

using namespace tabi;

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

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// bump allocator over the arena (256-byte aligned pieces)
struct Carve {
  char *base;
  size_t cap, used = 0;
  bool ok = true;
  template <typename T>
  T *take(size_t count) {
    const size_t bytes = round256(count * sizeof(T));
    if (used + bytes > cap) {
      ok = false;
      return nullptr;
    }
    T *p = reinterpret_cast<T *>(base + used);
    used += bytes;
    return p;
  }
};

bool valid_params(const tabi_params *p) {
  return p && p->version == TABI_PARAMS_VERSION && p->gutter >= 0 && p->gutter <= kMaxGutter &&
         p->knee_abs_pct >= 0 && p->knee_abs_pct <= 100 && p->knee_rel_pct >= 0 &&
         p->knee_rel_pct <= 100 && p->lr_sig_pct >= 0 && p->lr_sig_pct <= 100 &&
         p->knee_margin >= 0 && p->knee_margin <= 1 << 20 &&
         (p->flags & ~(TABI_F_ALL | TABI_F_EVAL_ALL)) == 0 && p->scale_fanout >= 0 &&
         p->scale_fanout <= kScales &&
         (p->laabb_count == 2 || p->laabb_count == 5 || p->laabb_count == kSlices) &&
         p->topt_permille >= 0 && p->topt_permille <= 1000 && p->hybrid_min_charts >= 0;
}

// Host <-> device copies of a batch's request arrays.  When the caller's
// host buffers are pinned (or registered), one kernel reads them (and,
// after the pack, writes the placements back) directly over the host link,
// instead of two copy calls per request in and one out; each copy is cut
// into pieces of at most kPieceBytes so that the CTAs share the large
// ones.  Buffers that the device cannot address (pageable memory) keep the
// copy calls.
constexpr uint64_t kPieceBytes = 64 * 1024;
struct CopyPiece {
  const uint8_t *src;
  uint8_t *dst;
  uint64_t bytes;
};

size_t pieces_of(uint64_t bytes) { return (size_t)((bytes + kPieceBytes - 1) / kPieceBytes); }

// Every piece starts kPieceBytes (a multiple of 16) into its copy, so a
// piece is 16-byte aligned at both ends iff its copy is; request arrays
// are 4-byte aligned (checked on the host).
__global__ void __launch_bounds__(256) copy_pieces_kernel(const CopyPiece *__restrict__ pcs, int n) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const CopyPiece pc = pcs[i];
    if ((((uintptr_t)pc.src | (uintptr_t)pc.dst) & 15) == 0) {
      const uint64_t n16 = pc.bytes >> 4;
      const uint4 *s = reinterpret_cast<const uint4 *>(pc.src);
      uint4 *d = reinterpret_cast<uint4 *>(pc.dst);
      for (uint64_t k = threadIdx.x; k < n16; k += blockDim.x) d[k] = s[k];
      for (uint64_t k = (n16 << 4) + threadIdx.x * 4; k < pc.bytes; k += blockDim.x * 4)
        *reinterpret_cast<uint32_t *>(pc.dst + k) = *reinterpret_cast<const uint32_t *>(pc.src + k);
    } else {
      for (uint64_t k = threadIdx.x * 4; k < pc.bytes; k += blockDim.x * 4)
        *reinterpret_cast<uint32_t *>(pc.dst + k) = *reinterpret_cast<const uint32_t *>(pc.src + k);
    }
  }
}

// `host` itself when the device can address that host buffer at the same
// address (pinned or registered memory under unified addressing) and it is
// 4-byte aligned; else null (the buffer then takes a copy call).
const void *device_view(const void *host) {
  if (((uintptr_t)host & 3) != 0) return nullptr;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost && a.devicePointer == host ? host : nullptr;
}

void add_pieces(std::vector<CopyPiece> &v, const void *src, void *dst, uint64_t bytes) {
  for (uint64_t o = 0; o < bytes; o += kPieceBytes)
    v.push_back(CopyPiece{static_cast<const uint8_t *>(src) + o, static_cast<uint8_t *>(dst) + o,
                          bytes - o < kPieceBytes ? bytes - o : kPieceBytes});
}

// Arena bytes of the per-chart and per-atlas arrays of one atlas (all but
// the envelope pools), with the host-input copies.
size_t fixed_bytes(int64_t n, int64_t nv) {
  const size_t per_chart = 4 + sizeof(tabi_chart_info) + 2 * sizeof(ChartShape) + 3 * 4 + 16 + 40 +
                           (size_t)kScales * (4 + 4 + 16 + 4 + 1 + 16) + 4 + 4 + 16 + sizeof(tabi_placement);
  const size_t per_atlas = sizeof(AtlasDesc) + (size_t)kScales * 2 * 8 * 2 + sizeof(ScaleOut) * kScales +
                           8 + sizeof(PackResult) + 8 + 40 * 256 + (size_t)kScales * (kCtlSave * 4 + 16) + 8;
  const size_t pieces = pieces_of(4 * (uint64_t)(n + 1)) + pieces_of(8 * (uint64_t)nv) +
                        pieces_of(sizeof(tabi_placement) * (uint64_t)n);
  return (size_t)n * per_chart + 8 * (size_t)nv + per_atlas + sizeof(CopyPiece) * pieces + 256 + sizeof(Pack) +
         64 * 1024;
}

// ---------------------------------------------------------------------------
// per-atlas kernels of the batch record
// ---------------------------------------------------------------------------
__global__ void init_kernel(const Pack *__restrict__ pp) {
  const Pack &p = *pp;
  const int t = threadIdx.x;
  if (blockIdx.x == 0) {
    if (t < 2 * kScales) p.jtot[t] = 0;
    for (int i = t; i < kScales * kChunkSlots; i += blockDim.x) {
      p.counter[i] = 0;
      p.rcounter[i] = 0;
    }
    if (t == 0) {
      *p.cur_wave = 0;
      p.raster_words[0] = p.raster_words[1] = 0;
    }
  }
  for (int at = blockIdx.x; at < p.A; at += gridDim.x) {
    if (t < kScales) p.scale_out[at * kScales + t] = ScaleOut{};
    if (t == 0) {
      p.found[at] = -1;
      p.err[at] = 0;
      p.area2[at] = 0;
      p.ext_sum[at] = 0;
      p.result[at] = PackResult{0, 0, 0, -1};
    }
    const int cb = p.atl[at].cb, n = p.atl[at].n;
    for (int s = t; s < n; s += blockDim.x) p.catl[cb + s] = at;
  }
}

// Per atlas: the successful candidate (Sec. 3.1 / Sec. 5) whose
// area-weighted mean scale is largest (Sec. 4.4; without a prefix-sum tail
// that is the largest successful candidate; ties keep the larger one), then
// its placements gathered back into input order, each with its chart's
// scale (the candidate's, or the tail's k').
__global__ void select_kernel(const Pack *__restrict__ pp) {
  __shared__ int best;
  __shared__ uint32_t err;
  const Pack &p = *pp;
  for (int at = blockIdx.x; at < p.A; at += gridDim.x) {
    if (threadIdx.x == 0) {
      int b = -1;
      unsigned __int128 bw = 0;
      for (int j = kScales - 1; j >= 0; --j) {
        const ScaleOut &so = p.scale_out[at * kScales + j];
        if (!so.success) continue;
        const unsigned __int128 w = ((unsigned __int128)so.wsum[1] << 64) | so.wsum[0];
        if (b < 0 || w > bw) { b = j; bw = w; }
      }
      best = b;
      err = p.err[at];
      PackResult r{0, 0, err, b};
      if (err & kErrInvalid) r.status = TABI_ERR_INVALID_ARG;
      else if (err & (kErrPool | kErrRow)) r.status = TABI_ERR_OOM;
      else if (b < 0) r.status = TABI_ERR_NO_FIT;
      else { r.status = TABI_OK; r.k = 16 * (b + 1); }
      p.result[at] = r;
    }
    __syncthreads();
    if (best >= 0 && !err) {
      const AtlasDesc &ad = p.atl[at];
      const int4 *place = p.place + (int64_t)best * p.N;
      const ScaleOut &so = p.scale_out[at * kScales + best];
      const int32_t kb = 16 * (best + 1), t0 = so.tail_start, kt = so.tail_k;
      for (int s = ad.cb + threadIdx.x; s < ad.cb + ad.n; s += blockDim.x) {
        const int c = p.perm[s];
        const int4 pl = place[s];
        const tabi_chart_info &inf = p.info[c];
        tabi_placement o;
        o.x = pl.x;
        o.y = pl.y;
        o.rot90 = (uint8_t)inf.rot90;
        o.flip_x = (uint8_t)inf.flip_x;
        o.flip_y = (uint8_t)inf.flip_y;
        o.mirror = (uint8_t)(pl.w & 1);
        o.k = s - ad.cb >= t0 ? kt : kb;
        ad.out[c - ad.cb] = o;
      }
    }
    __syncthreads();
  }
}

// Event pairs around each stage: (stage, start event, end event)
struct StageMarks {
  tabi_ctx *c;
  cudaStream_t st;
  int used = 0;
  static constexpr int kMax = tabi_ctx::kStageMarks;
  int stage[kMax];
  void begin(int s) {
    if (used >= kMax) return;
    stage[used] = s;
    cudaEventRecord(c->ev[2 * used], st);
  }
  void end() {
    if (used >= kMax) return;
    cudaEventRecord(c->ev[2 * used + 1], st);
    ++used;
  }
  void collect() {
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

int waves_of(int F) { return (kScales + F - 1) / F; }

// The launch sequence of a batch: prep, sort, layout, then descending waves
// of F candidates per atlas from its top candidate, each in Q chunks of the
// sorted charts (plan, raster, compaction, row loop), then selection.  The
// wave index lives in device memory; each wave ends with wave_end.
void enqueue_prologue(const Pack *dp, const Launch &L, cudaStream_t st, StageMarks *mk) {
  if (mk) mk->begin(0);
  launch_init(dp, L, st);
  launch_prep(dp, L, st);
  if (mk) { mk->end(); mk->begin(1); }
  launch_sort(dp, L, st);
  if (mk) { mk->end(); mk->begin(2); }
  launch_layout(dp, L, st);
  if (mk) mk->end();
}

void enqueue_wave(const Pack *dp, const Launch &L, int F, cudaStream_t st, StageMarks *mk,
                  cudaGraphConditionalHandle h, bool in_graph) {
  auto b = [&](int s) { if (mk) mk->begin(s); };
  auto e = [&]() { if (mk) mk->end(); };
  for (int q = 0; q < L.Q; ++q) {  // chart chunks of the wave (lazy evaluation)
    b(2);  // the wave plan counts with the layout
    launch_plan(dp, L, q, st);
    e();
    b(3);
    launch_raster(dp, L, q, F, st);
    e();
    b(4);
    launch_hcompact(dp, L, q, F, st);
    e();
    b(5);
    launch_rowloop(dp, L, q, F, st);
    e();
  }
  if (L.tail) {  // the prefix-sum tail (Sec. 4.4): its scale, redraw, push (with the row loop's time)
    b(5);
    for (int r = 0; r < tail_rounds(F); ++r) {
      launch_tail_round(dp, L, F, r, st);
      launch_rowloop(dp, L, L.Q, F, st);
    }
    e();
  }
  launch_wave_end(dp, h, in_graph, st);
}

void enqueue_select(const Pack *dp, const Launch &L, cudaStream_t st, StageMarks *mk) {
  if (mk) mk->begin(6);
  launch_select(dp, L, st);
  if (mk) mk->end();
}

// Direct launches (per-stage timing): every wave from the host.
void enqueue(const Pack *dp, const Launch &L, int F, cudaStream_t st, StageMarks *mk) {
  enqueue_prologue(dp, L, st, mk);
  for (int wave = 0; wave < waves_of(F); ++wave) enqueue_wave(dp, L, F, st, mk, 0, false);
  enqueue_select(dp, L, st, mk);
}

// The graph of a launch shape: prologue, a WHILE node whose body is one wave
// (wave_end decides on the device whether another wave runs, so waves in
// which no atlas searches cost nothing), then selection.
tabi_status capture_graph(tabi_ctx *ctx, const Launch &L, int F, cudaGraph_t *out) {
  const Pack *dp = reinterpret_cast<const Pack *>(ctx->arena);
  cudaStream_t s0 = ctx->cap_stream, s1 = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s1, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamCreate");
  cudaGraph_t graph = nullptr, body = nullptr;
  cudaGraphNode_t node = nullptr;
  cudaGraphConditionalHandle h = 0;
  bool capturing = false;
  const char *what = "cudaStreamBeginCapture";
  do {
    if ((e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) break;
    capturing = true;
    enqueue_prologue(dp, L, s0, nullptr);
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edges = nullptr;
    size_t ndeps = 0;
    what = "cudaStreamGetCaptureInfo";
    if ((e = cudaStreamGetCaptureInfo(s0, &cs, nullptr, &graph, &deps, &edges, &ndeps)) != cudaSuccess) break;
    what = "cudaGraphConditionalHandleCreate";
    if ((e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault)) != cudaSuccess) break;
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    what = "cudaGraphAddNode";
    if ((e = cudaGraphAddNode(&node, graph, deps, edges, ndeps, &np)) != cudaSuccess) break;
    body = np.conditional.phGraph_out[0];
    what = "cudaStreamUpdateCaptureDependencies";
    if ((e = cudaStreamUpdateCaptureDependencies(s0, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
      break;
    what = "body capture";
    if ((e = cudaStreamBeginCaptureToGraph(s1, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
      break;
    enqueue_wave(dp, L, F, s1, nullptr, h, true);
    cudaGraph_t body_out = nullptr;
    if ((e = cudaStreamEndCapture(s1, &body_out)) != cudaSuccess) break;
    enqueue_select(dp, L, s0, nullptr);
    what = "cudaStreamEndCapture";
    capturing = false;
    e = cudaStreamEndCapture(s0, &graph);
  } while (false);
  if (capturing) {
    cudaGraph_t junk = nullptr;
    cudaStreamEndCapture(s0, &junk);
    if (junk) cudaGraphDestroy(junk);
    graph = nullptr;
  }
  cudaStreamDestroy(s1);
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(ctx, e, what);
  }
  *out = graph;
  return TABI_OK;
}

tabi_status get_graph(tabi_ctx *ctx, const Launch &L, int F, cudaGraphExec_t *out) {
  for (const GraphEntry &g : ctx->graphs)
    if (g.F == F && g.smem == L.rowloop_smem && g.threads == L.rowloop_threads && g.ctas == L.rowloop_ctas &&
        g.Q == L.Q && g.prep_group == L.prep_group && g.laabb_k == L.laabb_k && g.tail == L.tail &&
        g.gutter == L.gutter) {
      *out = g.exec;
      return TABI_OK;
    }
  cudaGraph_t graph = nullptr;
  const tabi_status cs = capture_graph(ctx, L, F, &graph);
  if (cs != TABI_OK) return cs;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
  ctx->graphs.push_back(
      GraphEntry{F, L.rowloop_smem, L.rowloop_threads, L.rowloop_ctas, L.Q, L.prep_group, L.laabb_k, L.tail, L.gutter,
                 exec});
  *out = exec;
  return TABI_OK;
}

int ceil_log2(int64_t v) {
  int b = 0;
  while (((int64_t)1 << b) < v) ++b;
  return b;
}

// Batch class for the tuning cache: atlas count, mean chart count and
// widest atlas (powers of two), gutter, method flags and local-AABB count.
uint64_t batch_class(int A, int64_t N, int maxW, const tabi_params *params) {
  return (uint64_t)ceil_log2(A) | (uint64_t)ceil_log2((N + A - 1) / A) << 8 | (uint64_t)ceil_log2(maxW) << 16 |
         (uint64_t)params->gutter << 24 | (uint64_t)(params->flags & TABI_F_ALL) << 32 |
         (uint64_t)params->laabb_count << 40 | (uint64_t)(params->topt_permille > 0) << 44;
}

// One atlas: every candidate at once, no chunks and no progressive area
// bound (its successful candidate's row loop is the critical path, which
// stopping the failing ones early does not shorten); a batch: waves of
// eight candidates in four chunks, failing candidates stopped early.
Tuning default_tuning(int A) {
  return A == 1 ? Tuning{kScales, 32768, 1024, 1, 1, 0} : Tuning{8, 32768, 1024, 1, 4, 1};
}

bool ensure_hstage(tabi_ctx *ctx, size_t bytes) {
  if (ctx->hstage_bytes >= bytes) return true;
  if (ctx->hstage) cudaFreeHost(ctx->hstage);
  ctx->hstage = nullptr;
  ctx->hstage_bytes = 0;
  const size_t want = std::max(bytes, (size_t)1 << 16);
  if (cudaMallocHost(&ctx->hstage, want) != cudaSuccess) return false;
  ctx->hstage_bytes = want;
  return true;
}

// Host checks of one request; "" if it may run.
std::string check_request(const tabi_request &r, const tabi_params *params, int smem_dyn, bool host) {
  if (r.n_charts < 1 || r.n_charts > TABI_MAX_CHARTS) return "chart count outside [1, TABI_MAX_CHARTS]";
  if (r.n_verts < 3) return "fewer than 3 vertices";
  if (r.atlas_w < 1 || r.atlas_h < 1 || r.atlas_w > kMaxAtlas || r.atlas_h > kMaxAtlas)
    return "atlas side outside [1, 8192]";
  if (!r.offsets || !r.verts || !r.out) return "null pointer";
  if (rowloop_smem_bytes(r.atlas_w, params->gutter) > (size_t)smem_dyn)
    return "atlas too wide for this gutter: the row working set exceeds shared memory";
  if (host && (r.offsets[0] != 0 || r.offsets[r.n_charts] != (uint32_t)r.n_verts))
    return "offsets must run from 0 to n_verts";
  return "";
}

}  // namespace

// First half of a batch: host checks, arena carving, input copies, the
// launch sequence (graph replay) and the copies of the results into pinned
// staging, all enqueued on `stream`.  Nothing waits for the device (except
// with stage timing on).  The caller holds the context and calls
// batch_finish once the stream has reached this point.
tabi_status batch_launch(tabi_ctx *ctx, const tabi_params *params, tabi_request *reqs, int32_t R, void *stream,
                         bool host, const Tuning *force, Tuning *used, InFlight &fl, bool check) {
  fl = InFlight{};
  if (!valid_params(params)) return fail(ctx, TABI_ERR_INVALID_ARG, "bad params");
  if (!reqs || R < 1 || R > TABI_MAX_BATCH) return fail(ctx, TABI_ERR_INVALID_ARG, "bad request list");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");

  // host checks; the atlases that run, largest first (the row-loop queue
  // takes their tasks in this order)
  std::vector<int> &order = fl.order;
  std::string &first_error = fl.first_error;
  for (int r = 0; r < R; ++r) {
    reqs[r].scale_k = 0;
    reqs[r].status = TABI_ERR_INVALID_ARG;
    const std::string why = check_request(reqs[r], params, ctx->rowloop_dyn_max, host);
    if (why.empty()) order.push_back(r);
    else if (first_error.empty()) first_error = why;
  }
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return reqs[a].n_charts > reqs[b].n_charts; });
  const int A = (int)order.size();
  fl.A = A;
  ctx->has_last = false;
  if (A == 0) return TABI_OK;
  int64_t N = 0;
  for (int i = 0; i < A; ++i) N += reqs[order[i]].n_charts;
  if (N > 0x7fffffffLL) return fail(ctx, TABI_ERR_INVALID_ARG, "too many charts in one batch");

  // arena: the batch record first (its address is what the graphs read)
  Carve cv{ctx->arena, ctx->arena_bytes};
  Pack p{};
  Pack *dpack = cv.take<Pack>(1);
  AtlasDesc *ddesc = cv.take<AtlasDesc>(A);
  // copy pieces of the host buffers the device can address, in then out
  // (uploaded with the record: they follow the atlas table)
  size_t max_pieces = 0;
  if (host)
    for (int i = 0; i < A; ++i) {
      const tabi_request &r = reqs[order[i]];
      max_pieces += pieces_of(4 * ((uint64_t)r.n_charts + 1)) + pieces_of(8 * (uint64_t)r.n_verts) +
                    pieces_of(sizeof(tabi_placement) * (uint64_t)r.n_charts);
    }
  CopyPiece *dpieces = max_pieces ? cv.take<CopyPiece>(max_pieces) : nullptr;
  std::vector<AtlasDesc> &desc = fl.desc;
  desc.assign(A, AtlasDesc{});
  int64_t cb = 0;
  for (int i = 0; i < A; ++i) {
    const tabi_request &r = reqs[order[i]];
    AtlasDesc &d = desc[i];
    d.n = r.n_charts;
    d.nv = r.n_verts;
    d.W = r.atlas_w;
    d.H = r.atlas_h;
    d.cb = (int32_t)cb;
    d.pad = 0;
    cb += r.n_charts;
    if (host) {
      d.offsets = cv.take<uint32_t>((size_t)r.n_charts + 1);
      d.verts = cv.take<int32_t>(2 * (size_t)r.n_verts);
      d.out = cv.take<tabi_placement>((size_t)r.n_charts);
    } else {
      d.offsets = r.offsets;
      d.verts = r.verts;
      d.out = r.out;
    }
  }
  p.A = A;
  p.N = (int32_t)N;
  p.g = params->gutter;
  p.knee_abs = params->knee_abs_pct;
  p.knee_rel = params->knee_rel_pct;
  p.lr_sig = params->lr_sig_pct;
  p.knee_margin = params->knee_margin;
  p.flags = params->flags;
  p.laabb_k = params->laabb_count;
  p.topt = params->topt_permille;
  p.hyb_min = params->hybrid_min_charts;
  p.tail = 0;
  for (int i = 0; i < A && p.topt > 0; ++i) p.tail |= desc[i].n > p.hyb_min;
  // launch shape: forced (autotuner), else tuned for this batch class,
  // else the default; an explicit fan-out in params wins over both
  int maxW = 1;
  for (int i = 0; i < A; ++i) maxW = std::max(maxW, desc[i].W);
  const uint64_t cls = batch_class(A, N, maxW, params);
  Tuning tn = default_tuning(A);
  if (force) {
    tn = *force;
  } else {
    for (const TuneEntry &te : ctx->tuned)
      if (te.key == cls) tn = te.t;
    if (params->scale_fanout > 0) tn.F = params->scale_fanout;
  }
  p.F = tn.F;
  p.nwaves = waves_of(p.F);
  p.raster_items = tn.items;
  p.Q = tn.Q < 1 ? 1 : (tn.Q > kMaxChunks ? kMaxChunks : tn.Q);
  p.prog_bound = tn.B ? 1 : 0;
  p.wps_stride = 4;
  p.prep_group = prep_group_for(p.N, ctx->sms);
  for (int i = 0; i < A; ++i) p.wps_stride = std::max(p.wps_stride, (desc[i].W + 2 * p.g + 3) & ~3);
  p.atl = ddesc;
  const size_t n = (size_t)N;
  p.catl = cv.take<int32_t>(n);
  p.info = cv.take<tabi_chart_info>(n);
  p.shape_in = cv.take<ChartShape>(n);
  p.shape = cv.take<ChartShape>(n);
  p.perm = cv.take<int32_t>(n);
  p.hq = cv.take<int32_t>(n);
  p.wq = cv.take<int32_t>(n);
  p.sort_tmp = cv.take<uint32_t>(4 * n);
  p.colstart = cv.take<int32_t>(kScales * n);
  p.rowstart = cv.take<int32_t>(kScales * n);
  p.abase = cv.take<int64_t>((size_t)A * kScales * 2);
  p.atot = cv.take<int64_t>((size_t)A * kScales * 2);
  p.jtot = cv.take<unsigned long long>(kScales * 2);
  p.meta = cv.take<int32_t>(kScales * 4 * n);
  p.dnext = cv.take<int32_t>(kScales * n);
  p.pflags = cv.take<uint8_t>(kScales * n);
  p.place = cv.take<int4>(kScales * n);
  p.scale_out = cv.take<ScaleOut>((size_t)A * kScales);
  p.area2 = cv.take<unsigned long long>(A);
  p.ext_sum = cv.take<unsigned long long>(A);
  p.jtop = cv.take<int32_t>(A);
  p.found = cv.take<int32_t>(A);
  p.err = cv.take<uint32_t>(A);
  p.result = cv.take<PackResult>(A);
  p.act_info = cv.take<int32_t>(2);
  p.act_atl = cv.take<int32_t>(A);
  p.act_pre = cv.take<int32_t>(A);
  p.act_ext = cv.take<int4>(n);
  p.counter = cv.take<int32_t>(kScales * kChunkSlots);
  p.rcounter = cv.take<uint32_t>(kScales * kChunkSlots);
  p.cur_wave = cv.take<int32_t>(1);
  p.raster_words = cv.take<unsigned long long>(2);
  p.carea = cv.take<unsigned long long>(n);
  p.barea = cv.take<unsigned long long>(n);
  p.pre2 = cv.take<unsigned long long>(n);
  p.preE = cv.take<unsigned long long>(n);
  p.prea = cv.take<unsigned long long>(n);
  p.area_tot = cv.take<unsigned long long>(A);
  p.tstate = cv.take<int32_t>((size_t)A * kScales);
  p.front_save = cv.take<int32_t>((size_t)A * p.F * p.wps_stride);
  p.ctl_save = cv.take<int32_t>((size_t)A * p.F * kCtlSave);
  p.ttask = cv.take<int4>((size_t)A * p.F);
  p.tcount = cv.take<int32_t>(1);
  if (!cv.ok) return fail(ctx, TABI_ERR_OOM, "arena too small for the per-chart arrays");
  // the rest in equal thirds: column words, their chart indices, row words
  const size_t left = (cv.cap - cv.used) / sizeof(uint32_t);
  p.col_cap = p.row_cap = (int64_t)(left / 3) & ~(int64_t)63;
  if (p.col_cap < 64) return fail(ctx, TABI_ERR_OOM, "arena too small for the envelope pools");
  p.colpool = reinterpret_cast<uint32_t *>(cv.base + cv.used);
  p.colown = reinterpret_cast<int32_t *>(p.colpool + p.col_cap);
  p.pool = reinterpret_cast<uint32_t *>(p.colown + p.col_cap);

  // host buffers: pieces for those the device addresses, copy calls for
  // the rest (outputs: `out_call` marks the requests that need one)
  std::vector<CopyPiece> pin, pout;
  std::vector<char> in_call(host ? A : 0, 0), out_call(host ? A : 0, 0);
  for (int i = 0; i < A && host; ++i) {
    const tabi_request &r = reqs[order[i]];
    const uint64_t bo = 4 * ((uint64_t)r.n_charts + 1), bv = 8 * (uint64_t)r.n_verts;
    const void *so = device_view(r.offsets), *sv = device_view(r.verts);
    if (so && sv) {
      add_pieces(pin, so, (void *)desc[i].offsets, bo);
      add_pieces(pin, sv, (void *)desc[i].verts, bv);
    } else {
      in_call[i] = 1;
    }
    void *dout = const_cast<void *>(device_view(r.out));
    if (dout) add_pieces(pout, desc[i].out, dout, sizeof(tabi_placement) * (uint64_t)r.n_charts);
    else out_call[i] = 1;
  }

  // the record, the atlas table and the copy pieces go up in one copy
  const size_t desc_off = round256(sizeof(Pack));
  const size_t pcs_off = desc_off + round256(sizeof(AtlasDesc) * (size_t)A);
  const size_t npcs = pin.size() + pout.size();
  const size_t up = npcs ? pcs_off + sizeof(CopyPiece) * npcs : desc_off + sizeof(AtlasDesc) * (size_t)A;
  const size_t res_off = round256(up);
  if (npcs && (!dpieces || reinterpret_cast<char *>(dpieces) != reinterpret_cast<char *>(dpack) + pcs_off ||
               npcs > max_pieces))
    return fail(ctx, TABI_ERR_CUDA, "copy pieces misplaced");  // cannot happen: the carve is contiguous
  // with the overlap counter: its atlas table (up) and counts (down)
  const size_t chk_tab = round256(res_off + sizeof(PackResult) * (size_t)A);
  const size_t chk_cnt = round256(chk_tab + sizeof(CheckAtlas) * (size_t)A);
  const size_t stage_end = check ? chk_cnt + 24 * (size_t)A : res_off + sizeof(PackResult) * (size_t)A;
  if (!ensure_hstage(ctx, stage_end)) return fail(ctx, TABI_ERR_CUDA, "pinned staging allocation failed");
  memcpy(ctx->hstage, &p, sizeof(Pack));
  memcpy(ctx->hstage + desc_off, desc.data(), sizeof(AtlasDesc) * (size_t)A);
  if (npcs) {
    memcpy(ctx->hstage + pcs_off, pin.data(), sizeof(CopyPiece) * pin.size());
    memcpy(ctx->hstage + pcs_off + sizeof(CopyPiece) * pin.size(), pout.data(), sizeof(CopyPiece) * pout.size());
  }
  e = cudaMemcpyAsync(dpack, ctx->hstage, up, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !pin.empty()) {
    copy_pieces_kernel<<<ctx->sms * 4, 256, 0, st>>>(dpieces, (int)pin.size());
    e = cudaGetLastError();
  }
  for (int i = 0; i < A && host && e == cudaSuccess; ++i) {
    if (!in_call[i]) continue;
    const tabi_request &r = reqs[order[i]];
    e = cudaMemcpyAsync((void *)desc[i].offsets, r.offsets, sizeof(uint32_t) * ((size_t)r.n_charts + 1),
                        cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((void *)desc[i].verts, r.verts, sizeof(int32_t) * 2 * (size_t)r.n_verts,
                          cudaMemcpyHostToDevice, st);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "input copy");

  // the row-loop CTA's shared memory: what the widest atlas wants, in
  // 16 KiB classes (fewer graphs), at most what the device allows
  size_t want = 0;
  for (int i = 0; i < A; ++i) want = std::max(want, rowloop_smem_wanted(desc[i].W, p.g));
  int smem = (int)((want + 16383) & ~(size_t)16383);
  if (smem > ctx->rowloop_dyn_max) smem = ctx->rowloop_dyn_max;
  Launch L{ctx->sms, smem, tn.threads == 512 ? 512 : 1024, 1, p.Q, p.prep_group, p.laabb_k, p.tail != 0, p.g};
  if (L.rowloop_threads == 512 && tn.ctas == 2) {
    // two CTAs per multiprocessor if both fit its shared memory
    const int two = (ctx->smem_per_sm - 2 * (ctx->smem_reserved + rowloop_static_smem())) / 2 & ~255;
    if ((int)want <= two) {
      L.rowloop_smem = std::min(smem, two);
      L.rowloop_ctas = 2;
    }
  }
  if (used) *used = Tuning{tn.F, tn.items, L.rowloop_threads, L.rowloop_ctas, p.Q, p.prog_bound};
  if (ctx->timing) {
    StageMarks mk{ctx, st};
    enqueue(dpack, L, p.F, st, &mk);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pack");
    mk.collect();
  } else {
    cudaGraphExec_t exec = nullptr;
    const tabi_status gs = get_graph(ctx, L, p.F, &exec);
    if (gs != TABI_OK) return gs;
    cudaEventRecord(ctx->tev[0], st);
    e = cudaGraphLaunch(exec, st);
    cudaEventRecord(ctx->tev[1], st);
    fl.timed = true;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphLaunch");
  }
  if (check) {
    // App. B's overlap and gutter counts of every atlas, behind the pack:
    // the table, the counts and the bit planes in the (now free) envelope
    // pools; an atlas whose planes do not fit is left unchecked
    char *pools = reinterpret_cast<char *>(p.colpool);
    const size_t pool_bytes = 3 * (size_t)p.col_cap * sizeof(uint32_t);
    const size_t tab_bytes = round256(sizeof(CheckAtlas) * (size_t)A), cnt_bytes = round256(24 * (size_t)A);
    const size_t scr_bytes = check_scratch_bytes(p.N);
    CheckAtlas *htab = reinterpret_cast<CheckAtlas *>(ctx->hstage + chk_tab);
    int64_t words = 0;
    const size_t fixed = tab_bytes + cnt_bytes + scr_bytes;
    const int64_t cap = pool_bytes > fixed ? (int64_t)((pool_bytes - fixed) / 4) : -1;
    for (int i = 0; i < A; ++i) {
      CheckAtlas &ca = htab[i];
      fill_check_atlas(ca, desc[i].W, desc[i].H, p.g);
      ca.offsets = desc[i].offsets;
      ca.verts = desc[i].verts;
      ca.place = desc[i].out;
      ca.n = desc[i].n;
      ca.cb = desc[i].cb;
      ca.pad = 0;
      const int64_t need = check_plane_words(desc[i].W, desc[i].H, p.g);
      ca.plane0 = cap >= 0 && words + need <= cap ? words : -1;
      if (ca.plane0 >= 0) words += need;
    }
    CheckAtlas *dtab = reinterpret_cast<CheckAtlas *>(pools);
    unsigned long long *dcnt = reinterpret_cast<unsigned long long *>(pools + tab_bytes);
    void *scratch = pools + tab_bytes + cnt_bytes;
    uint32_t *planes = reinterpret_cast<uint32_t *>(pools + fixed);
    if (!ctx->cev[0]) {
      cudaEventCreate(&ctx->cev[0]);
      cudaEventCreate(&ctx->cev[1]);
    }
    cudaEventRecord(ctx->cev[0], st);
    e = cudaMemcpyAsync(dtab, htab, sizeof(CheckAtlas) * (size_t)A, cudaMemcpyHostToDevice, st);
    if (cap < 0) {  // no room for the charts' scratch: the batch stays unchecked
      if (e == cudaSuccess) e = cudaMemsetAsync(dcnt, 0xff, 24 * (size_t)A, st);
    } else {
      if (e == cudaSuccess) e = cudaMemsetAsync(dcnt, 0, 24 * (size_t)A, st);
      if (e == cudaSuccess) {
        launch_check(dtab, A, p.catl, p.N, p.g, planes, words, scratch, dcnt, ctx->sms, st);
        e = cudaGetLastError();
      }
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ctx->hstage + chk_cnt, dcnt, 24 * (size_t)A, cudaMemcpyDeviceToHost, st);
    cudaEventRecord(ctx->cev[1], st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "overlap check");
    fl.checked = true;
    fl.check_off = chk_cnt;
  }
  PackResult *hres = reinterpret_cast<PackResult *>(ctx->hstage + res_off);
  e = cudaMemcpyAsync(hres, p.result, sizeof(PackResult) * (size_t)A, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && !pout.empty()) {
    copy_pieces_kernel<<<ctx->sms * 4, 256, 0, st>>>(dpieces + pin.size(), (int)pout.size());
    e = cudaGetLastError();
  }
  for (int i = 0; i < A && host && e == cudaSuccess; ++i) {
    if (!out_call[i]) continue;
    const tabi_request &r = reqs[order[i]];
    e = cudaMemcpyAsync(r.out, desc[i].out, sizeof(tabi_placement) * (size_t)r.n_charts,
                        cudaMemcpyDeviceToHost, st);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "result copy");
  fl.p = p;
  fl.res_off = res_off;
  return TABI_OK;
}

// Second half: after the stream has passed batch_launch's work, the
// per-request statuses and the inspection state.
tabi_status batch_finish(tabi_ctx *ctx, tabi_request *reqs, int32_t R, InFlight &fl, float *ms_out) {
  if (fl.A == 0) {
    ctx->last_error = fl.first_error;
    return TABI_OK;
  }
  if (ms_out && fl.timed) cudaEventElapsedTime(ms_out, ctx->tev[0], ctx->tev[1]);
  const PackResult *hres = reinterpret_cast<const PackResult *>(ctx->hstage + fl.res_off);
  ctx->last = fl.p;
  ctx->last_desc = fl.desc;
  ctx->last_map.assign(R, -1);
  for (int i = 0; i < fl.A; ++i) {
    tabi_request &r = reqs[fl.order[i]];
    ctx->last_map[fl.order[i]] = i;
    r.status = hres[i].status;
    r.scale_k = hres[i].status == TABI_OK ? hres[i].k : 0;
  }
  ctx->has_last = true;
  ctx->last_error = fl.first_error;
  return TABI_OK;
}

void batch_quality(tabi_ctx *ctx, const InFlight &fl, int r, int64_t out[3]) {
  out[0] = out[1] = out[2] = -1;
  if (!fl.checked || r < 0 || r >= (int)ctx->last_map.size() || ctx->last_map[r] < 0) return;
  const unsigned long long *c = reinterpret_cast<const unsigned long long *>(ctx->hstage + fl.check_off);
  const int i = ctx->last_map[r];
  for (int q = 0; q < 3; ++q) out[q] = c[3 * i + q] == ~0ull ? -1 : (int64_t)c[3 * i + q];
}

namespace {

// One batch, synchronously; the caller holds the context.
tabi_status run_batch_locked(tabi_ctx *ctx, const tabi_params *params, tabi_request *reqs, int32_t R,
                             void *stream, bool host, const Tuning *force = nullptr, float *ms_out = nullptr,
                             Tuning *used = nullptr) {
  InFlight fl;
  tabi_status s = batch_launch(ctx, params, reqs, R, stream, host, force, used, fl);
  if (s != TABI_OK || fl.A == 0) {
    if (s == TABI_OK) batch_finish(ctx, reqs, R, fl, nullptr);
    return s;
  }
  const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pack");
  return batch_finish(ctx, reqs, R, fl, ms_out);
}

tabi_status run_batch(tabi_ctx *ctx, const tabi_params *params, tabi_request *reqs, int32_t R, void *stream,
                      bool host) {
  if (!ctx) return TABI_ERR_INVALID_ARG;
  Guard guard(ctx);
  if (!guard.ok) return fail(ctx, TABI_ERR_BUSY, "context in use");
  return run_batch_locked(ctx, params, reqs, R, stream, host);
}

tabi_status run_single(tabi_ctx *ctx, const tabi_params *params, int32_t W, int32_t H, int32_t n,
                       const uint32_t *offsets, const int32_t *verts, int32_t nv, tabi_placement *out,
                       int32_t *out_k, void *stream, bool host) {
  if (!ctx) return TABI_ERR_INVALID_ARG;
  if (!out_k) return fail(ctx, TABI_ERR_INVALID_ARG, "null out_k");
  *out_k = 0;
  tabi_request r{W, H, n, nv, offsets, verts, out, 0, 0};
  const tabi_status s = run_batch(ctx, params, &r, 1, stream, host);
  if (s != TABI_OK) return s;
  *out_k = r.scale_k;
  switch (r.status) {
    case TABI_OK: return TABI_OK;
    case TABI_ERR_NO_FIT: return fail(ctx, TABI_ERR_NO_FIT, "no candidate scale fits every chart");
    case TABI_ERR_INVALID_ARG:
      if (ctx->has_last) return fail(ctx, TABI_ERR_INVALID_ARG, "invalid chart (vertices, size or range)");
      return TABI_ERR_INVALID_ARG;  // host check; last_error says which
    default: return fail(ctx, TABI_ERR_OOM, "arena too small for the envelopes of this input");
  }
}

}  // namespace

namespace tabi {
void launch_init(const Pack *dp, const Launch &L, cudaStream_t st) {
  init_kernel<<<L.sms * 2, 256, 0, st>>>(dp);
}
void launch_select(const Pack *dp, const Launch &L, cudaStream_t st) {
  select_kernel<<<L.sms * 2, 256, 0, st>>>(dp);
}
}  // namespace tabi

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
  p->laabb_count = kSlices;
  p->topt_permille = 10;        // Sec. 4.4: t_opt = 1 % ...
  p->hybrid_min_charts = 10000;  // ... for atlases of more than 10,000 charts
  p->scale_fanout = 0;  // tuned, else 64 for one atlas and 8 for a batch
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
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  // the row loop's dynamic shared memory may use all the opt-in space
  // beyond its static part; raise the limit once so every graph can launch
  cudaDeviceGetAttribute(&c->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
  cudaDeviceGetAttribute(&c->smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, device);
  const int stat = rowloop_static_smem();
  c->rowloop_dyn_max = stat < 0 ? 0 : (optin - stat) & ~255;
  bool ok = c->sms > 0 && c->rowloop_dyn_max > 0 && rowloop_prepare(c->rowloop_dyn_max) == cudaSuccess &&
            cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreate(&c->tev[0]) == cudaSuccess && cudaEventCreate(&c->tev[1]) == cudaSuccess;
  if (ok && arena) {
    c->arena = (char *)arena;
  } else if (ok) {
    ok = cudaMalloc(&c->arena, arena_bytes) == cudaSuccess;
    c->owned = ok;
  }
  if (!ok) {
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (cudaEvent_t ev : c->tev)
      if (ev) cudaEventDestroy(ev);
    delete c;
    return TABI_ERR_CUDA;
  }
  *out = c;
  return TABI_OK;
}

void tabi_ctx_destroy(tabi_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  for (GraphEntry &g : c->graphs) cudaGraphExecDestroy(g.exec);
  for (int i = 0; i < c->n_ev; ++i) cudaEventDestroy(c->ev[i]);
  for (cudaEvent_t ev : c->tev)
    if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : c->cev)
    if (ev) cudaEventDestroy(ev);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->owned) cudaFree(c->arena);
  if (c->hstage) cudaFreeHost(c->hstage);
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
    case TABI_PENDING: return "pending";
  }
  return "unknown status";
}

size_t tabi_arena_bytes(int32_t n, int32_t nv, int32_t W, int32_t H, int64_t sum_extent_texels,
                        int32_t gutter) {
  (void)W; (void)H;
  if (n < 1) return 0;
  // column words, their chart indices and row words get equal shares; at
  // candidate k each must hold the larger of sum(w') and sum(h'), both at
  // most sum_extent * k / 1024 + n (2g + 2) (+ 3 alignment words), and the
  // 64 candidates of one wave together at most 64 times the k = 1024 sizes
  const size_t pool = (size_t)kScales * 4 * 3 *
                      ((size_t)sum_extent_texels + (size_t)n * (2 * (size_t)gutter + 2) + 4);
  return fixed_bytes(n, nv) + pool + (size_t)kScales * 256;
}

tabi_status tabi_pack(tabi_ctx *ctx, const tabi_params *params, int32_t W, int32_t H, int32_t n,
                      const uint32_t *offsets, const int32_t *verts, int32_t nv, tabi_placement *out,
                      int32_t *out_k, void *stream) {
  return run_single(ctx, params, W, H, n, offsets, verts, nv, out, out_k, stream, true);
}

tabi_status tabi_pack_device(tabi_ctx *ctx, const tabi_params *params, int32_t W, int32_t H,
                             int32_t n, const uint32_t *offsets, const int32_t *verts, int32_t nv,
                             tabi_placement *out, int32_t *out_k, void *stream) {
  return run_single(ctx, params, W, H, n, offsets, verts, nv, out, out_k, stream, false);
}

tabi_status tabi_pack_batch(tabi_ctx *ctx, const tabi_params *params, tabi_request *reqs, int32_t n_reqs,
                            void *stream) {
  return run_batch(ctx, params, reqs, n_reqs, stream, true);
}

tabi_status tabi_pack_batch_device(tabi_ctx *ctx, const tabi_params *params, tabi_request *reqs,
                                   int32_t n_reqs, void *stream) {
  return run_batch(ctx, params, reqs, n_reqs, stream, false);
}

tabi_status tabi_pack_batch_shaped(tabi_ctx *ctx, const tabi_params *params, tabi_request *reqs,
                                   int32_t n_reqs, void *stream, int32_t device_pointers,
                                   const tabi_tuning *shape) {
  if (!ctx) return TABI_ERR_INVALID_ARG;
  if (!shape) return fail(ctx, TABI_ERR_INVALID_ARG, "null shape");
  if (shape->scale_fanout < 1 || shape->scale_fanout > kScales || shape->raster_warp_items < 1 ||
      (shape->rowloop_threads != 512 && shape->rowloop_threads != 1024) || shape->rowloop_ctas < 1 ||
      shape->rowloop_ctas > 2 || shape->chunks < 1 || shape->chunks > kMaxChunks ||
      (shape->progressive_bound != 0 && shape->progressive_bound != 1))
    return fail(ctx, TABI_ERR_INVALID_ARG, "bad launch shape");
  Guard guard(ctx);
  if (!guard.ok) return fail(ctx, TABI_ERR_BUSY, "context in use");
  const Tuning t{shape->scale_fanout, shape->raster_warp_items, shape->rowloop_threads, shape->rowloop_ctas,
                 shape->chunks, shape->progressive_bound};
  return run_batch_locked(ctx, params, reqs, n_reqs, stream, device_pointers == 0, &t);
}

tabi_status tabi_autotune(tabi_ctx *ctx, const tabi_params *params, tabi_request *reqs, int32_t n_reqs,
                          void *stream, tabi_tuning *out) {
  if (!ctx) return TABI_ERR_INVALID_ARG;
  Guard guard(ctx);
  if (!guard.ok) return fail(ctx, TABI_ERR_BUSY, "context in use");
  if (ctx->timing) return fail(ctx, TABI_ERR_INVALID_ARG, "stage timing is on");
  // coordinate search from the default shape: fan-out, then raster
  // warp-items, then the row-loop CTA shape; each candidate timed on its
  // second run (the first captures its graph).  A shape under which some
  // atlas ends differently (an arena too small for a wide wave) is out.
  Tuning best = default_tuning(n_reqs);
  float best_ms = -1.f;
  std::vector<int32_t> ref;
  auto trial = [&](const Tuning &t) -> tabi_status {
    float ms = 0.f, ms2 = 0.f;
    Tuning used{};
    tabi_status s = run_batch_locked(ctx, params, reqs, n_reqs, stream, false, &t, &ms, &used);
    if (s == TABI_OK) s = run_batch_locked(ctx, params, reqs, n_reqs, stream, false, &t, &ms2, &used);
    if (s != TABI_OK) return s;
    if (!ctx->has_last) return fail(ctx, TABI_ERR_INVALID_ARG, "no request passed the host checks");
    std::vector<int32_t> got(n_reqs);
    for (int i = 0; i < n_reqs; ++i) got[i] = reqs[i].status;
    if (ref.empty()) ref = got;
    if (got != ref) return TABI_OK;
    if (best_ms < 0.f || ms2 < best_ms) { best_ms = ms2; best = used; }
    return TABI_OK;
  };
  {
    const tabi_status s = trial(best);
    if (s != TABI_OK) return s;
  }
  const int fanouts[] = {kScales, 16, 8, 4, 2, 1};
  const Tuning start = best;
  for (int F : fanouts) {
    if (F == start.F) continue;
    Tuning t = start;
    t.F = F;
    const tabi_status s = trial(t);
    if (s != TABI_OK) return s;
  }
  const int items[] = {16384, 65536};
  const Tuning base = best;
  for (int it : items) {
    Tuning t = base;
    t.items = it;
    const tabi_status s = trial(t);
    if (s != TABI_OK) return s;
  }
  {
    Tuning t = best;
    t.threads = 512;
    t.ctas = 2;
    const tabi_status s = trial(t);
    if (s != TABI_OK) return s;
  }
  {  // the other chunkings: all charts at once, or lazily in four, six or eight chunks
    const Tuning base_q = best;
    for (int Q : {1, 4, 6, 8}) {
      if (Q == base_q.Q) continue;
      Tuning t = base_q;
      t.Q = Q;
      const tabi_status s = trial(t);
      if (s != TABI_OK) return s;
    }
  }
  {  // the progressive area bound on or off
    Tuning t = best;
    t.B = !best.B;
    const tabi_status s = trial(t);
    if (s != TABI_OK) return s;
  }
  {  // leave the requests with the chosen shape's results
    float ms = 0.f;
    const tabi_status s = run_batch_locked(ctx, params, reqs, n_reqs, stream, false, &best, &ms, nullptr);
    if (s != TABI_OK) return s;
  }
  // remember it for this batch class (tabi_params.scale_fanout = 0 uses it)
  const Pack &p = ctx->last;
  int maxW = 1;
  for (const AtlasDesc &d : ctx->last_desc) maxW = std::max(maxW, d.W);
  const uint64_t cls = batch_class(p.A, p.N, maxW, params);
  bool found = false;
  for (TuneEntry &te : ctx->tuned)
    if (te.key == cls) { te.t = best; te.ms = best_ms; found = true; }
  if (!found) ctx->tuned.push_back(TuneEntry{cls, best, best_ms});
  if (out) {
    out->scale_fanout = best.F;
    out->raster_warp_items = best.items;
    out->rowloop_threads = best.threads;
    out->rowloop_ctas = best.ctas;
    out->chunks = best.Q;
    out->progressive_bound = best.B;
    out->ms = best_ms;
  }
  return TABI_OK;
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

tabi_status tabi_inspect_atlas(tabi_ctx *ctx, int32_t atlas, int32_t what, int32_t scale, void *dst,
                               size_t cap, size_t *needed) {
  if (!ctx || !ctx->has_last || !needed) return TABI_ERR_INVALID_ARG;
  Guard g(ctx);
  if (!g.ok) return fail(ctx, TABI_ERR_BUSY, "context in use");
  if (atlas < 0 || atlas >= (int)ctx->last_map.size() || ctx->last_map[atlas] < 0)
    return fail(ctx, TABI_ERR_INVALID_ARG, "no such atlas in the last batch");
  if (scale < 0 || scale >= kScales) return fail(ctx, TABI_ERR_INVALID_ARG, "bad scale index");
  cudaSetDevice(ctx->device);
  const Pack &p = ctx->last;
  const int at = ctx->last_map[atlas];
  const AtlasDesc &ad = ctx->last_desc[at];
  const size_t n = (size_t)ad.n;
  const int64_t js = (int64_t)scale * p.N + ad.cb;
  // region starts and sizes of this atlas (small reads, needed to size ENV),
  // then its top candidate
  int64_t reg[2 * kScales * 2 + 5];
  cudaError_t e = cudaMemcpy(reg, p.abase + region(at, 0, 0), sizeof(int64_t) * 2 * kScales,
                             cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(reg + 2 * kScales, p.atot + region(at, 0, 0), sizeof(int64_t) * 2 * kScales,
                   cudaMemcpyDeviceToHost);
  int32_t jt = 0, waves = 0;
  unsigned long long rwords[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(&jt, p.jtop + at, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&waves, p.cur_wave, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(rwords, p.raster_words, sizeof(rwords), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "inspect copy");
  reg[4 * kScales] = jt;
  reg[4 * kScales + 1] = waves;
  reg[4 * kScales + 2] = p.prep_group;
  reg[4 * kScales + 3] = (int64_t)rwords[0];
  reg[4 * kScales + 4] = (int64_t)rwords[1];
  const int64_t words[2] = {reg[2 * kScales + 2 * scale], reg[2 * kScales + 2 * scale + 1]};
  struct Piece {
    const void *src;
    size_t bytes;
    bool host;
  };
  Piece pcs[5] = {};
  bool local_perm = false;
  switch (what) {
    case TABI_INSPECT_CHARTS: pcs[0] = {p.info + ad.cb, sizeof(tabi_chart_info) * n, false}; break;
    case TABI_INSPECT_PERM: pcs[0] = {p.perm + ad.cb, 4 * n, false}; local_perm = true; break;
    case TABI_INSPECT_ENV:
      if (scale > jt) return fail(ctx, TABI_ERR_INVALID_ARG, "candidate above the area bound's top: no envelopes");
      pcs[0] = {words, sizeof(words), true};
      pcs[1] = {p.meta + js * 4, 16 * n, false};
      pcs[2] = {p.rowstart + js, 4 * n, false};
      pcs[3] = {p.colpool + reg[2 * scale], 4 * (size_t)words[0], false};
      pcs[4] = {p.pool + reg[2 * scale + 1], 4 * (size_t)words[1], false};
      break;
    case TABI_INSPECT_REGIONS: pcs[0] = {reg, sizeof(reg), true}; break;
    case TABI_INSPECT_PAIRS:
      pcs[0] = {p.dnext + js, 4 * n, false};
      pcs[1] = {p.pflags + js, n, false};
      break;
    case TABI_INSPECT_SCALE:
      pcs[0] = {p.scale_out + at * kScales + scale, sizeof(ScaleOut), false};
      pcs[1] = {p.place + js, 16 * n, false};
      break;
    default: return fail(ctx, TABI_ERR_INVALID_ARG, "bad inspect selector");
  }
  *needed = 0;
  for (const Piece &pc : pcs) *needed += pc.bytes;
  if (!dst || cap < *needed) return fail(ctx, TABI_ERR_INVALID_ARG, "buffer too small");
  char *d = (char *)dst;
  for (const Piece &pc : pcs) {
    if (!pc.bytes) continue;
    if (pc.host) {
      memcpy(d, pc.src, pc.bytes);
    } else {
      e = cudaMemcpy(d, pc.src, pc.bytes, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "inspect copy");
    }
    d += pc.bytes;
  }
  if (local_perm) {  // sorted position -> input index within the atlas
    int32_t *pm = (int32_t *)dst;
    for (size_t s = 0; s < n; ++s) pm[s] -= ad.cb;
  }
  return TABI_OK;
}

tabi_status tabi_check_packing_device(tabi_ctx *ctx, int32_t W, int32_t H, int32_t gutter, int32_t n,
                                      const uint32_t *offsets, const int32_t *verts, int32_t nv,
                                      const tabi_placement *place, tabi_quality *out, void *stream) {
  if (!ctx) return TABI_ERR_INVALID_ARG;
  if (!out || !offsets || !verts || !place || n < 1 || nv < 3 || W < 1 || H < 1 || W > kMaxAtlas ||
      H > kMaxAtlas || gutter < 0 || gutter > kMaxGutter)
    return fail(ctx, TABI_ERR_INVALID_ARG, "bad check arguments");
  Guard guard(ctx);
  if (!guard.ok) return fail(ctx, TABI_ERR_BUSY, "context in use");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  const cudaStream_t st = (cudaStream_t)stream;
  const int64_t words = check_plane_words(W, H, gutter);
  const size_t scr_bytes = check_scratch_bytes(n);
  if (512 + scr_bytes + (size_t)words * 4 > ctx->arena_bytes)
    return fail(ctx, TABI_ERR_OOM, "arena too small for the check");
  if (!ensure_hstage(ctx, 512)) return fail(ctx, TABI_ERR_CUDA, "pinned staging allocation failed");
  ctx->has_last = false;  // the arena is reused: the last pack can no longer be inspected
  CheckAtlas *h = reinterpret_cast<CheckAtlas *>(ctx->hstage);
  fill_check_atlas(*h, W, H, gutter);
  h->offsets = offsets;
  h->verts = verts;
  h->place = place;
  h->n = n;
  h->cb = 0;
  h->pad = 0;
  h->plane0 = 0;
  CheckAtlas *dtab = reinterpret_cast<CheckAtlas *>(ctx->arena);
  unsigned long long *dcnt = reinterpret_cast<unsigned long long *>(ctx->arena + 256);
  void *scratch = ctx->arena + 512;
  uint32_t *planes = reinterpret_cast<uint32_t *>(ctx->arena + 512 + scr_bytes);
  unsigned long long *hcnt = reinterpret_cast<unsigned long long *>(ctx->hstage + 256);
  e = cudaMemcpyAsync(dtab, h, sizeof(CheckAtlas), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dcnt, 0, 24, st);
  if (e == cudaSuccess) {
    launch_check(dtab, 1, nullptr, n, gutter, planes, words, scratch, dcnt, ctx->sms, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(hcnt, dcnt, 24, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "overlap check");
  out->overlap_texels = (int64_t)hcnt[0];
  out->gutter_texels = (int64_t)hcnt[1];
  out->outside_texels = (int64_t)hcnt[2];
  return TABI_OK;
}

tabi_status tabi_inspect(tabi_ctx *ctx, int32_t what, int32_t scale, void *dst, size_t cap, size_t *needed) {
  return tabi_inspect_atlas(ctx, 0, what, scale, dst, cap, needed);
}

}  // extern "C"
