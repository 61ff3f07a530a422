// Internal declarations of the GB300 packer: device records, launch helpers.
// Integer conventions are those of include/tabi.h (Q.8 vertices, k/1024
// scales, 2^-18-texel scaled coordinates).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tabi.h"

namespace tabi {

constexpr int kSlices = 10;          // local AABBs per axis (App. A; Tab. 13 default)
constexpr int kAngles = 8;           // OBB rotations m*pi/16, m = 0..7 (App. A)
constexpr int kScales = 64;          // candidates k = 16*(j+1), j = 0..63 (Sec. 5)
constexpr int kMaxAtlas = 8192;      // atlas side limit (front fits shared memory)
constexpr int kMaxGutter = 8;
constexpr int64_t kFix = 1LL << 18;  // scaled units per texel (Q.8 * k)

// Error bits raised by kernels into Pack::err.
enum : uint32_t { kErrInvalid = 1u, kErrPool = 2u, kErrRow = 4u };

// Scale-independent shape record of one chart, in sorted order (what the
// envelope rasterizer reads).  32-byte aligned for vector loads.
struct __align__(16) ChartShape {
  int32_t Wq, Hq, m, pad;
  int64_t u0, u1, v0, v1;
  int32_t tlo[kSlices], bhi[kSlices], llo[kSlices], rhi[kSlices];
};

// Per-candidate-scale summary (TABI_INSPECT_SCALE header).
struct ScaleOut {
  int32_t success, rows, knee_rows, knees, score, placed, evaluated, pad;
};

// Result of one pack, written on the device and read once by the host.
struct PackResult {
  int32_t status;  // tabi_status
  int32_t k;
  uint32_t err;
  int32_t best_j;
};

// Everything one pack needs on the device; pointers into the arena.
struct Pack {
  int32_t n, nv, W, H, g;
  int32_t knee_abs, knee_rel, lr_sig, knee_margin;
  uint32_t flags;
  const uint32_t *offsets;
  const int32_t *verts;
  tabi_chart_info *info;   // [n] input order
  ChartShape *shape_in;    // [n] input order
  ChartShape *shape;       // [n] sorted order
  int32_t *perm;           // [n] sorted position -> input index
  int32_t *hq;             // [n] sorted Hq (Q.8)
  uint32_t *sort_tmp;      // [4n] radix-sort ping-pong
  int32_t *env_off;        // [2n] row-pool offset and row capacity (sizes at k = 1024)
  int32_t *colstart;       // [64 * n] column-pool offset of each chart at each candidate
  int64_t col_stride;      // uint32 column entries per candidate scale
  int64_t row_stride;      // uint32 row entries per candidate scale
  uint32_t *colpool;       // [64 * col_stride] Top' | Bot' << 16, charts back to back
  int32_t *colown;         // [64 * col_stride] sorted chart index of each column word
  uint32_t *pool;          // [64 * row_stride] L' | R' << 16, k = 1024 capacities
  int32_t *meta;           // [64 * 4n]: w', h', column start, max bottom
  int32_t *dnext;          // [64 * n]  compacting distance (s, s+1)
  uint8_t *pflags;         // [64 * n]  interlock bits
  int4 *place;             // [64 * n]  x, y, row, bits
  ScaleOut *scale_out;     // [64]
  int32_t *found;          // highest successful candidate index so far (-1 none)
  PackResult *result;
  uint32_t *err;
  tabi_placement *out;     // [n] input order
};

// Launch helpers (each .cu file owns its kernels).  All are asynchronous on
// `st`; `j_hi` .. `j_lo` is a descending block of candidate indices.
void launch_prep(const Pack &p, cudaStream_t st);
void launch_sort(const Pack &p, cudaStream_t st);
void launch_layout(const Pack &p, cudaStream_t st);
void launch_raster(const Pack &p, int j_lo, int j_hi, cudaStream_t st);
void launch_hcompact(const Pack &p, int j_lo, int j_hi, cudaStream_t st);
cudaError_t launch_rowloop(const Pack &p, int j_lo, int j_hi, cudaStream_t st);
size_t rowloop_smem_bytes(int W, int g);  // shared memory one row-loop CTA needs
void launch_select(const Pack &p, cudaStream_t st);
void launch_init(const Pack &p, cudaStream_t st);

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

// OBB angle table (App. A: 8 rotations evenly spaced in [0, 7*pi/16]):
// C_m = round-half-away(2^14 * cos(m*pi/16)), S_m likewise with sin.
static __constant__ int32_t kObbCos[kAngles] = {16384, 16069, 15137, 13623, 11585, 9102, 6270, 3196};
static __constant__ int32_t kObbSin[kAngles] = {0, 3196, 6270, 9102, 11585, 13623, 15137, 16069};

}  // namespace tabi
