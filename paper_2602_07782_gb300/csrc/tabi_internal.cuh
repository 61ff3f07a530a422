// Internal declarations of the GB300 packer: device records, launch helpers.
// Integer conventions are those of include/tabi.h (Q.8 vertices, k/1024
// scales, 2^-18-texel scaled coordinates).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tabi.h"
#include "raster_math.cuh"

namespace tabi {

constexpr int kSlices = 10;          // most local AABBs per axis (App. A default; Tab. 13 also 2, 5)
constexpr int kAngles = 8;           // OBB rotations m*pi/16, m = 0..7 (App. A)
constexpr int kScales = 64;          // candidates k = 16*(j+1), j = 0..63 (Sec. 5)
constexpr int kMaxAtlas = 8192;      // atlas side limit (front fits shared memory)
constexpr int kMaxGutter = 8;
constexpr int64_t kFix = 1LL << 18;  // scaled units per texel (Q.8 * k)

// Error bits raised by kernels into Pack::err (one word per atlas).
enum : uint32_t { kErrInvalid = 1u, kErrPool = 2u, kErrRow = 4u };

// Scale-independent shape record of one chart, in sorted order (what the
// envelope rasterizer reads).  32-byte aligned for vector loads.  Slot t of
// the slice arrays holds slice floor(t K / 10) of K: ylo/yhi the extremes
// of y over the x-slice, xlo/xhi those of x over the y-slice (Q.8).
struct __align__(16) ChartShape {
  int32_t Wq, Hq, m, pad;
  int64_t u0, u1, v0, v1;
  int32_t ylo[kSlices], yhi[kSlices], xlo[kSlices], xhi[kSlices];
};

// Per-(atlas, candidate scale) summary (TABI_INSPECT_SCALE header).
// evaluated: 0 not run, 1 ran to its end, 2 abandoned once the candidate
// could no longer win.  The prefix-sum tail (Sec. 4.4): its rows, its
// scale k' (0: none, or none fitted) and its first chart (n: no tail).
// wsum: sum over the charts of twice the area (Q.8^2) times the chart's
// scale (the area-weighted mean scale times the total), set on success.
struct ScaleOut {
  int32_t success, rows, knee_rows, knees, score, placed, evaluated, tail_rows;
  int32_t tail_k, tail_start, pad0, pad1;
  unsigned long long wsum[2];  // low, high 64 bits
};

// Row-loop task state of an (atlas, candidate) per wave: 0 running (or not
// begun), 1 finished, 2 prefix-sum tail folded at the candidate scale and
// waiting for its intermediate scale, 3 searched: the tail rows wait to be
// pushed at that scale (or, if none fitted, the rows to go on one by one).
enum : int32_t { kTaskRun = 0, kTaskDone = 1, kTaskTailSearch = 2, kTaskTailPush = 3 };
// A tail chart's place record between the fold and the push: (0, 0, tail
// row, row length | kTailFirst) for the first chart of a row, (0, 0, tail
// row, 0) for the others.
constexpr int32_t kTailFirst = 0x40000000;
// ints per parked row-loop state (ctl_save)
constexpr int kCtlSave = 32;
// fields of a parked state used by the tail
enum : int {
  kCsTail = 10, kCsC0 = 15, kCsHeadRows = 16, kCsTrows = 17, kCsLo = 18, kCsHi = 19, kCsMask = 20,
  kCsRound = 21, kCsKt = 22, kCsCommitted = 23
};

// Result of one atlas, written on the device and read once by the host.
struct PackResult {
  int32_t status;  // tabi_status
  int32_t k;
  uint32_t err;
  int32_t best_j;
};

// One atlas of a batch: its inputs and output (device pointers) and where
// its charts sit in the batch's chart index space [cb, cb + n).
struct AtlasDesc {
  const uint32_t *offsets;  // [n + 1] CSR over this atlas's vertices
  const int32_t *verts;     // [2 nv] x, y pairs, Q.8
  tabi_placement *out;      // [n] input order
  int32_t n, nv, W, H;
  int32_t cb, pad;
};

// Everything a batch of packs needs on the device.  The record itself lives
// in device memory (kernels take a pointer to it), so one captured launch
// sequence serves every batch with the same wave structure.
//
// Chart indices are global over the batch: atlas a owns input and sorted
// positions [cb_a, cb_a + n_a).  Per-candidate arrays are [64][N].
struct Pack {
  int32_t A, N;                 // atlases, charts over all atlases
  int32_t g, knee_abs, knee_rel, lr_sig, knee_margin;
  uint32_t flags;
  int32_t F;                    // candidates per wave (scale fan-out)
  int32_t nwaves;
  int32_t raster_items;         // target warp-items of a raster wave
  int32_t Q;                    // chart chunks per wave (1: all charts at once)
  int32_t wps_stride;           // ints per saved frontline (widest atlas, padded)
  int32_t prep_group;           // prep lanes per chart (host record of the launch)
  int32_t prog_bound;           // row loop checks the progressive area bound after each row
  int32_t laabb_k;              // local AABBs per axis (2, 5 or 10; record slot t holds slice t K / 10)
  int32_t topt;                 // t_opt of the prefix-sum tail, permille of the atlas height (0: off)
  int32_t hyb_min;              // the tail applies to atlases of more charts than this
  int32_t tail;                 // some atlas of the batch may take the tail (the launch sequence has its kernels)
  const AtlasDesc *atl;         // [A]
  int32_t *catl;                // [N] atlas of each chart
  tabi_chart_info *info;        // [N] input order
  ChartShape *shape_in;         // [N] input order
  ChartShape *shape;            // [N] sorted order
  int32_t *perm;                // [N] sorted position -> input index
  int32_t *hq, *wq;             // [N] sorted Hq, Wq (Q.8)
  uint32_t *sort_tmp;           // [4N] radix-sort ping-pong
  int32_t *colstart;            // [64 N] column offset inside the (atlas, candidate) region
  int32_t *rowstart;            // [64 N] row offset inside the (atlas, candidate) region
  int64_t *abase;               // [A][64][2] column / row region start in the pools
  int64_t *atot;                // [A][64][2] column / row region words (multiples of 4)
  unsigned long long *jtot;     // [64][2] words of all atlases at rank r (candidate jtop - r)
  int64_t col_cap, row_cap;     // words per pool
  uint32_t *colpool;            // Top' | Bot' << 16 per padded column
  int32_t *colown;              // atlas-local sorted index of each column word
  uint32_t *pool;               // L' | R' << 16 per padded row
  int32_t *meta;                // [64 N][4]: w', h', column start, max bottom
  int32_t *dnext;               // [64 N] compacting distance (s, s+1)
  uint8_t *pflags;              // [64 N] interlock bits
  int4 *place;                  // [64 N] x, y, row, bits
  ScaleOut *scale_out;          // [A][64]
  unsigned long long *area2;    // [A] twice the summed area of the charts certified simple (Q.8^2)
  unsigned long long *ext_sum;  // [A] summed larger AABB side of the charts (Q.8)
  int32_t *jtop;                // [A] largest candidate the area bound allows (-1 none)
  int32_t *found;               // [A] highest successful candidate so far (-1 none)
  uint32_t *err;                // [A]
  PackResult *result;           // [A]
  int32_t *act_info;            // [2]: atlases still searching, their charts
  int32_t *act_atl;             // [A] those atlases, in batch order
  int32_t *act_pre;             // [A] their first position in act_ext
  int4 *act_ext;                // [N] their charts: chart (global sorted index), atlas, the
                                //     atlas's top candidate, its first chart | 1 << 31 for its last
  int32_t *counter;             // [64][kChunkSlots] row-loop task counter of each (wave, chunk; tail push)
  uint32_t *rcounter;           // [64][kChunkSlots] raster warp-item counter of each (wave, chunk)
  int32_t *cur_wave;            // the wave the kernels work on (advanced by wave_end)
  unsigned long long *raster_words;  // [2] padded scanline words / column words the raster evaluated
  unsigned long long *carea;    // [N] twice each chart's polygon area |shoelace| (Q.8^2), input order
  unsigned long long *barea;    // [N] carea if the loop is certified simple, else 0 (the area bounds)
  unsigned long long *pre2;     // [N] sorted order: barea summed over the atlas's earlier charts
  unsigned long long *preE;     // [N] sorted order: Hq summed over the atlas's earlier charts
  unsigned long long *prea;     // [N] sorted order: carea summed over the atlas's earlier charts
  unsigned long long *area_tot; // [A] carea summed over the atlas (the weights of Sec. 4.4's choice)
  int32_t *tstate;              // [A][64] row-loop task state (kTask*)
  int32_t *front_save;          // [A][F][wps_stride] frontline of a task between chunks
  int32_t *ctl_save;            // [A][F][kCtlSave] row state of a task between chunks (and its tail search)
  int4 *ttask;                  // [A F] tail tasks of the wave: atlas, candidate, slot, first tail chart
  int32_t *tcount;              // [1] how many
};

// One atlas for the overlap and gutter counter (check.cu): its charts
// (device pointers, input order), placements, size and gutter, and where
// its four bit planes start in the planes buffer (-1: no room, unchecked).
struct CheckAtlas {
  const uint32_t *offsets;
  const int32_t *verts;
  const tabi_placement *place;
  int32_t n, W, H, g;
  int32_t wpp, wpd;  // words per plain row (W bits), per padded row (W + 2g bits)
  int32_t cb, pad;   // first chart in the batch's chart index space
  int64_t plane0;
};
int64_t check_plane_words(int W, int H, int g);
void fill_check_atlas(CheckAtlas &ca, int W, int H, int g);
// Counts per atlas (3 x uint64: plain texels covered twice, dilated
// texels covered twice, cover texels outside the atlas; all ~0 when the
// atlas was not checked); counts must be zero on entry.  catl: the atlas
// of each of the N charts (NULL: all in atlas 0); gmax: the largest
// gutter of the atlases (sets the row masks' shared memory); scratch:
// check_scratch_bytes(N) bytes of device memory (256-byte aligned).
size_t check_scratch_bytes(int64_t N);
void launch_check(const CheckAtlas *datl, int A, const int32_t *catl, int64_t N, int gmax, uint32_t *planes,
                  int64_t words, void *scratch, unsigned long long *counts, int sms, cudaStream_t st);

// Region of (atlas a, candidate j) in the column / row pools.
__host__ __device__ __forceinline__ int64_t region(int a, int j, int which) {
  return ((int64_t)a * kScales + j) * 2 + which;
}

// Chart chunks of a wave (lazy evaluation, see the row loop): chunk q of an
// atlas of n sorted charts ends at ceil(n e_q / 64) with
//   Q = 1: e = 64;  Q = 2: e = 16, 64;  Q = 4: e = 8, 16, 32, 64;
//   Q = 6: e = 2, 8, 16, 24, 40, 64;  Q = 8: e = 1, 2, 4, 8, 16, 24, 40, 64
// (the first chunks are short -- the sorted charts come tallest first, and
// a candidate far above the answer fails within its first rows).
constexpr int kMaxChunks = 8;
constexpr int kChunkSlots = kMaxChunks + 1;  // per wave: the chunks, then the tail's push pass
__host__ __device__ __forceinline__ int chunk_end(int n, int q, int Q) {
  int e;
  switch (Q) {
    case 1: e = 64; break;
    case 2: e = q ? 64 : 16; break;
    case 4: e = 8 << q; break;
    case 6: { constexpr int t[6] = {2, 8, 16, 24, 40, 64}; e = t[q]; break; }
    default: { constexpr int t[8] = {1, 2, 4, 8, 16, 24, 40, 64}; e = t[q]; break; }
  }
  return q == Q - 1 ? n : (int)(((int64_t)n * e + 63) >> 6);
}

// Candidates of atlas a in wave w: ranks r = w F .. w F + F - 1 below the
// atlas's top candidate, i.e. j = jtop - r for the r with j >= 0.
struct WaveRange {
  int lo, hi;  // candidate indices lo .. hi (empty if hi < lo)
};
__host__ __device__ __forceinline__ WaveRange wave_range(int jtop, int wave, int F) {
  const int hi = jtop - wave * F;
  const int lo = hi - F + 1 < 0 ? 0 : hi - F + 1;
  return WaveRange{lo, hi};
}

// Launch helpers (each .cu file owns its kernels).  All are asynchronous on
// `st` and capturable; grids are fixed per device (persistent kernels loop
// over the device-side work), so they depend only on the wave structure.
struct Launch {
  int sms;             // multiprocessors
  int rowloop_smem;    // dynamic shared memory of a row-loop CTA
  int rowloop_threads; // 1024 or 512 threads per row-loop CTA
  int rowloop_ctas;    // row-loop CTAs per multiprocessor (512 threads: 1 or 2)
  int Q;               // chart chunks per wave
  int prep_group;      // prep lanes per chart: 32, 16, 8 or 4
  int laabb_k;         // local AABBs per axis: 2, 5 or 10 (selects the prep kernel)
  bool tail;           // the batch may take the prefix-sum tail: its kernels follow each wave
  int gutter;          // g (the tail's trial kernel picks its lane groups by it)
};
void launch_init(const Pack *dp, const Launch &L, cudaStream_t st);
void launch_prep(const Pack *dp, const Launch &L, cudaStream_t st);
int prep_group_for(int64_t charts, int sms);
void launch_sort(const Pack *dp, const Launch &L, cudaStream_t st);
void launch_layout(const Pack *dp, const Launch &L, cudaStream_t st);
void launch_plan(const Pack *dp, const Launch &L, int q, cudaStream_t st);
void launch_raster(const Pack *dp, const Launch &L, int q, int F, cudaStream_t st);
void launch_hcompact(const Pack *dp, const Launch &L, int q, int F, cudaStream_t st);
// Ends a wave: advances the wave index and, inside a captured graph, sets
// the loop condition (another wave iff an atlas can still search).
void launch_wave_end(const Pack *dp, cudaGraphConditionalHandle h, bool in_graph, cudaStream_t st);
cudaError_t rowloop_prepare(int smem);  // raise the CTA's shared-memory limit (not capturable)
int rowloop_static_smem();              // the row-loop kernel's static shared memory
void launch_rowloop(const Pack *dp, const Launch &L, int q, int F, cudaStream_t st);
void launch_select(const Pack *dp, const Launch &L, cudaStream_t st);
// The prefix-sum tail after a wave's last chunk (Sec. 4.4), in rounds: per
// round the largest parked tail tasks of each atlas (1, 2, 4, ..., then the
// rest), their trial scales, the redraw and the compaction at the chosen
// scale (the row loop's push pass follows each round).
int tail_rounds(int F);
void launch_tail_round(const Pack *dp, const Launch &L, int F, int round, cudaStream_t st);
constexpr int kTailRounds = 1;  // trial scales k - 14 .. k (one candidate step), one launch
constexpr int kTailSteps = 14;  // the tail's scale is at least k - 14
size_t rowloop_smem_bytes(int W, int g);       // shared memory a row-loop CTA needs without the stage
size_t rowloop_smem_wanted(int W, int g);      // ... with a stage of two atlas widths

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t b) {  // b > 0
  int64_t q = a / b;
  if ((a % b) != 0 && a < 0) --q;
  return q;
}
__device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) {  // b > 0
  int64_t q = a / b;
  if ((a % b) != 0 && a > 0) ++q;
  return q;
}
// floor / ceil of a / 2^18 (arithmetic shifts floor toward -inf)
__device__ __forceinline__ int64_t floor_fix(int64_t a) { return a >> 18; }
__device__ __forceinline__ int64_t ceil_fix(int64_t a) { return -((-a) >> 18); }

template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u < v ? u : v;
  }
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}

// Reductions inside an aligned group of G lanes of a warp (G a power of two,
// mask gm from group_mask<G>()).
template <int G, typename T>
__device__ __forceinline__ T group_min(T v, unsigned gm) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const T u = __shfl_xor_sync(gm, v, o);
    v = u < v ? u : v;
  }
  return v;
}
template <int G, typename T>
__device__ __forceinline__ T group_max(T v, unsigned gm) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const T u = __shfl_xor_sync(gm, v, o);
    v = u > v ? u : v;
  }
  return v;
}
template <int G>
__device__ __forceinline__ unsigned group_mask() {
  return G == 32 ? 0xffffffffu : (((1u << G) - 1) << (threadIdx.x & (32 - G)));
}

// Stable LSD radix sort of keys below 2^21 (three passes of 7-bit digits)
// by one CTA of kRadixThreads threads: on entry kA/vA hold n keys and their
// values, on exit kB/vB hold them sorted by increasing key, equal keys in
// their entry order (passes A -> B -> A -> B).  Each warp owns a contiguous
// run of the input; per pass a histogram [digit][warp] counts the digits
// (lanes with equal digits found by __match_any_sync, their leader adds
// the count), an exclusive scan in digit-major order gives every (digit,
// warp) its first output slot, and the scatter walks each run in order.
// The height sort of the pack (Sec. 3.1) and the allocation-free height
// sort both call this.
constexpr int kRadixThreads = 1024;
__device__ __forceinline__ void radix_sort21(uint32_t *kA, uint32_t *vA, uint32_t *kB, uint32_t *vB, int n) {
  constexpr int kW = kRadixThreads / 32, kDig = 128;
  __shared__ uint32_t hist[kDig * kW];  // [digit][warp]
  __shared__ uint32_t part[kW];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int chunk = ((n + kW - 1) / kW + 31) & ~31;
  const int beg = w * chunk, end = min(n, beg + chunk);
  const unsigned lt = (1u << lane) - 1u;
  __syncthreads();  // the caller's key fill is complete
  for (int pass = 0; pass < 3; ++pass) {
    const int shift = 7 * pass;
    const uint32_t *ks = (pass & 1) ? kB : kA, *vs = (pass & 1) ? vB : vA;
    uint32_t *kd = (pass & 1) ? kA : kB, *vd = (pass & 1) ? vA : vB;
    for (int i = tid; i < kDig * kW; i += kRadixThreads) hist[i] = 0;
    __syncthreads();
    for (int base = beg; base < end; base += 32) {
      const int i = base + lane;
      const bool ok = i < end;
      const uint32_t d = ok ? (ks[i] >> shift) & (kDig - 1) : kDig;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      if (ok && lane == __ffs(peers) - 1) hist[d * kW + w] += __popc(peers);
      __syncwarp();  // the next leader of this digit may be another lane
    }
    __syncthreads();
    // exclusive scan of hist in digit-major order (4 entries per thread)
    uint32_t loc[4], sum = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) { loc[q] = hist[tid * 4 + q]; sum += loc[q]; }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) part[w] = incl;
    __syncthreads();
    if (w == 0) {
      const uint32_t x = part[lane];
      uint32_t y = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += u;
      }
      part[lane] = y - x;
    }
    __syncthreads();
    uint32_t run = part[w] + incl - sum;
#pragma unroll
    for (int q = 0; q < 4; ++q) { hist[tid * 4 + q] = run; run += loc[q]; }
    __syncthreads();
    for (int base = beg; base < end; base += 32) {
      const int i = base + lane;
      const bool ok = i < end;
      const uint32_t key = ok ? ks[i] : 0u;
      const uint32_t d = ok ? (key >> shift) & (kDig - 1) : kDig;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      uint32_t dst = 0;
      if (ok) dst = hist[d * kW + w] + __popc(peers & lt);
      __syncwarp();
      if (ok && lane == __ffs(peers) - 1) hist[d * kW + w] += __popc(peers);
      __syncwarp();
      if (ok) { kd[dst] = key; vd[dst] = vs[i]; }
    }
    __syncthreads();
  }
}

// Sec. 4.4's choice among the successful candidates: the largest
// sum_c area_c * scale_c (wsum).  No chart's scale exceeds its candidate's,
// so once a candidate with sum w has succeeded, candidate j can only win if
// 16 (j + 1) * total > w: candidates below floor(w / (16 total)) are moot
// (all of them, if the charts have no area).  This is the atlas's `found`.
__device__ __forceinline__ int32_t moot_below(unsigned __int128 w, unsigned long long total) {
  if (total == 0) return kScales;
  const unsigned __int128 q = w / ((unsigned __int128)total * 16u);
  return q > (unsigned __int128)kScales ? kScales : (int32_t)q;
}

// Charts surely folded row by row at candidate k (Sec. 4.4): the tail only
// takes charts no taller than the first chart of its first row, which is
// shorter than t_opt H, so every chart with 1000 ceil(Hq k / 2^18) >=
// t_opt H is placed before it, at k; the others end at k or at the tail's
// scale, which is at least k - kTailSteps.  hq_sorted is the atlas's
// sorted Hq (non-increasing); returns how many such charts lead it (n
// when the tail cannot apply).
__host__ __device__ __forceinline__ int head_prefix(const int32_t *hq_sorted, int n, int64_t k, int topt, int H,
                                                    bool hybrid) {
  if (!hybrid) return n;
  int lo = 0, hi = n;  // first index whose chart is short enough for the tail
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int64_t h = ((int64_t)hq_sorted[mid] * k + kFix - 1) >> 18;
    if (1000 * h >= (int64_t)topt * H) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// OBB angle table (App. A: 8 rotations evenly spaced in [0, 7*pi/16]):
// C_m = round-half-away(2^14 * cos(m*pi/16)), S_m likewise with sin.
static __constant__ int32_t kObbCos[kAngles] = {16384, 16069, 15137, 13623, 11585, 9102, 6270, 3196};
static __constant__ int32_t kObbSin[kAngles] = {0, 3196, 6270, 9102, 11585, 13623, 15137, 16069};
// Magic numbers for exact division by the table entries (raster_math.cuh,
// fdiv_magic); sin 0 is never a divisor (m = 0 has no OBB constraint).
static __constant__ rmath::Magic kObbDivCos[kAngles] = {
    rmath::magic_div(16384), rmath::magic_div(16069), rmath::magic_div(15137), rmath::magic_div(13623),
    rmath::magic_div(11585), rmath::magic_div(9102),  rmath::magic_div(6270),  rmath::magic_div(3196)};
static __constant__ rmath::Magic kObbDivSin[kAngles] = {
    rmath::magic_div(2),     rmath::magic_div(3196),  rmath::magic_div(6270),  rmath::magic_div(9102),
    rmath::magic_div(11585), rmath::magic_div(13623), rmath::magic_div(15137), rmath::magic_div(16069)};

}  // namespace tabi
