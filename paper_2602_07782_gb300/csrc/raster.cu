// Envelope rasterizer (App. A "Parallel Pushing Algorithm", Sec. 4.1.2, Sec. 5
// gutters).
//
// For each candidate scale k/1024 and sorted chart, one warp produces
//   * per padded column i (w' = w + 2g of them): Top'(i) | Bot'(i) << 16,
//   * per padded row r (h' = h + 2g of them):   L'(r) | R'(r) << 16,
// packed as uint32 into that scale's envelope pool, plus the chart's padded
// size and maximum bottom.  One warp walks one chart through a run of
// consecutive candidates; for each it derives the chart's per-scale
// constants (local-AABB piece ranges, OBB line terms, and the corners, which
// are carried incrementally from candidate to candidate; see
// raster_math.cuh) lane-parallel into shared memory, then lane l of chunk t
// handles raw column 32t + l with 32-bit arithmetic.
// The gutter dilation min/max over raw columns i-2g..i takes the values from
// lanes l-o of the current chunk or, across the chunk seam, of the previous
// chunk (kept in registers), so each raw value is computed exactly once.
//
// Columns go to a per-candidate column pool with the charts back to back
// (the row loop copies a row's columns in one contiguous range); rows go to
// a row pool laid out once by the sizes at k = 1024 (the largest scale).
#include "raster_math.cuh"
#include "tabi_internal.cuh"

namespace tabi {
namespace {

constexpr int32_t kBig = 0x3fffffff;
constexpr int kRasterThreads = 256;
constexpr int kRasterWarps = kRasterThreads / 32;

// One axis of one chart: raw scanlines 0..len-1 from the per-warp constants,
// padded scanlines 0..len+2g-1 written to dst.  Returns max upper' (axis 0:
// the chart's deepest padded BottomEdge).
__device__ __forceinline__ int32_t warp_axis(const rmath::AxisK &ak, int g, uint32_t *__restrict__ dst) {
  const int lane = threadIdx.x & 31;
  const int32_t len = ak.len;
  const int32_t padded = len + 2 * g;
  int32_t prev_lo = kBig, prev_hi = -kBig;
  int32_t maxhi = 0;
  for (int32_t base = 0; base < padded; base += 32) {
    const int32_t c = base + lane;
    int32_t lo = kBig, hi = -kBig;
    if (c < len) rmath::scanline(ak, c, lo, hi);
    int32_t dlo = lo, dhi = hi;
    for (int o = 1; o <= 2 * g; ++o) {
      const int32_t clo = __shfl_sync(0xffffffffu, lo, (lane - o) & 31);
      const int32_t chi = __shfl_sync(0xffffffffu, hi, (lane - o) & 31);
      const int32_t plo = __shfl_sync(0xffffffffu, prev_lo, (lane - o) & 31);
      const int32_t phi = __shfl_sync(0xffffffffu, prev_hi, (lane - o) & 31);
      const int32_t vlo = lane >= o ? clo : plo, vhi = lane >= o ? chi : phi;
      dlo = vlo < dlo ? vlo : dlo;
      dhi = vhi > dhi ? vhi : dhi;
    }
    if (c < padded) {
      const int32_t hi2 = dhi + 2 * g;
      dst[c] = (uint32_t)dlo | ((uint32_t)hi2 << 16);
      maxhi = hi2 > maxhi ? hi2 : maxhi;
    }
    prev_lo = lo;
    prev_hi = hi;
  }
  return warp_max(maxhi);
}

__global__ void __launch_bounds__(kRasterThreads, 4) raster_kernel(Pack p, int j_lo, int nj, int G) {
  __shared__ rmath::AxisK axk[kRasterWarps][2];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t n = p.n;
  const int ngroups = (nj + G - 1) / G;
  if (gw >= n * ngroups) return;
  if (*(volatile int32_t *)p.found >= 0) return;  // a larger scale already succeeded
  if (*(volatile uint32_t *)p.err) return;        // invalid input or pool overflow: write nothing
  const int s = (int)(gw / ngroups);
  const int j0 = j_lo + (int)(gw % ngroups) * G;
  const int j1 = min(j0 + G, j_lo + nj);
  const ChartShape &sh = p.shape[s];
  const bool use_l = (p.flags & TABI_F_LAABB) != 0, use_o = (p.flags & TABI_F_OBB) != 0;
  const int m = sh.m;
  const int64_t C = kObbCos[m], S = kObbSin[m];
  const int32_t roff = p.env_off[2 * s];
  const int g = p.g;
  rmath::AxisK &a0 = axk[wib][0], &a1 = axk[wib][1];
  // lanes 24-31 carry the eight corner quantities across the candidates
  rmath::CornerQ cq;
  const bool corner_lane = lane >= 24 && use_o && m > 0;
  if (corner_lane) rmath::corner_init(cq, lane - 24, 16 * (j0 + 1), 16, C, S, sh.u0, sh.u1, sh.v0, sh.v1);
  for (int j = j0; j < j1; ++j) {
    const int64_t k = 16 * (j + 1);
    // per-(chart, scale) constants, lane-parallel: lanes 0-19 the local-AABB
    // pieces, lanes 20-21 the OBB line terms, lanes 24-31 the corners
    if (lane < 2 * rmath::kK) {
      const int ax = lane >= rmath::kK, i = lane - ax * rmath::kK;
      rmath::setup_piece(ax ? a1 : a0, i, ax ? sh.Hq : sh.Wq, k, ax ? sh.llo[i] : sh.tlo[i],
                         ax ? sh.rhi[i] : sh.bhi[i]);
    } else if (lane < 2 * rmath::kK + 2) {
      const int ax = lane - 2 * rmath::kK;
      rmath::setup_obb_base(ax ? a1 : a0, ax, sh.Wq, sh.Hq, k, m, C, S, sh.u0, sh.u1, sh.v0, sh.v1, use_l,
                            use_o);
    } else if (corner_lane) {
      rmath::corner_store(cq, lane - 24, (lane - 24) >> 2 ? a1 : a0);
      rmath::corner_advance(cq);
    }
    __syncwarp();
    const int32_t cstart = p.colstart[(int64_t)j * n + s];
    const int32_t maxbot = warp_axis(a0, g, p.colpool + (int64_t)j * p.col_stride + cstart);
    {  // each column word's chart, so a staged run of words knows its owners
      int32_t *own = p.colown + (int64_t)j * p.col_stride + cstart;
      for (int c = lane; c < a0.len + 2 * g; c += 32) own[c] = s;
    }
    warp_axis(a1, g, p.pool + (int64_t)j * p.row_stride + roff);
    if (lane == 0) {
      int32_t *mt = p.meta + ((int64_t)j * n + s) * 4;
      mt[0] = a0.len + 2 * g;
      mt[1] = a1.len + 2 * g;
      mt[2] = cstart;
      mt[3] = maxbot;
    }
    __syncwarp();
  }
}

// Pool layouts.  Block j < 64: column offsets of candidate j, charts back to
// back (exclusive scan of w'(k_j)), so any run of consecutive charts has its
// columns in one contiguous range.  Block 64: the row pool's offsets from
// the row counts at k = 1024, rounded to 16-byte segments, shared by every
// candidate (rows are only read per chart pair).
__global__ void __launch_bounds__(1024) layout_kernel(Pack p) {
  __shared__ int64_t part[32];
  __shared__ int64_t carry;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int j = blockIdx.x;
  const bool rows = j == kScales;
  const int64_t k = 16 * (j + 1);
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < p.n; base += 1024) {
    const int s = base + tid;
    int64_t sz = 0, cap = 0;
    if (s < p.n) {
      const ChartShape &sh = p.shape[s];
      if (rows) {
        cap = ((sh.Hq + 255) >> 8) + 2 * p.g;
        sz = (cap + 3) & ~3LL;
      } else {
        sz = ((sh.Wq * k + kFix - 1) >> 18) + 2 * p.g;
      }
    }
    int64_t incl = sz;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) part[w] = incl;
    __syncthreads();
    if (w == 0) {
      const int64_t x = part[lane];
      int64_t y = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += u;
      }
      part[lane] = y - x;
    }
    __syncthreads();
    const int64_t excl = carry + part[w] + incl - sz;
    if (s < p.n) {
      if (rows) {
        p.env_off[2 * s] = (int32_t)excl;
        p.env_off[2 * s + 1] = (int32_t)cap;
      } else {
        p.colstart[(int64_t)j * p.n + s] = (int32_t)excl;
      }
    }
    __syncthreads();
    if (tid == 1023) carry = excl + sz;
    __syncthreads();
  }
  if (tid == 0 && carry > (rows ? p.row_stride : p.col_stride)) atomicOr(p.err, kErrPool);
}

// ---------------------------------------------------------------------------
// horizontal compactor (Sec. 4.1.2, App. A interlock)
// ---------------------------------------------------------------------------
template <bool kMax>
__device__ __forceinline__ int32_t warp_scan_incl(int32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v = kMax ? (u > v ? u : v) : (u < v ? u : v);
  }
  return v;
}

// One warp per (scale, sorted pair (s, s+1)), A = s left of B = s+1,
// top-aligned:  d = w'_A - max_r (R'_A(r) - L'_B(r));  B may move up
// relative to A iff every row of B stays right of all rows of A above it;
// A may move up relative to B iff every row of A stays left of all rows of
// B above it.
__global__ void __launch_bounds__(256) hcompact_kernel(Pack p, int j_lo, int nj) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t n = p.n;
  if (gw >= n * nj) return;
  if (*(volatile int32_t *)p.found >= 0) return;
  if (*(volatile uint32_t *)p.err) return;
  const int j = j_lo + (int)(gw / n);
  const int s = (int)(gw % n);
  const int64_t ps = (int64_t)j * n + s;
  if (s == n - 1) {
    if (lane == 0) { p.dnext[ps] = 0; p.pflags[ps] = 0; }
    return;
  }
  const int32_t *ma = p.meta + ps * 4, *mb = ma + 4;
  const int32_t wA = ma[0], hA = ma[1], hB = mb[1];
  const uint32_t *pool = p.pool + (int64_t)j * p.row_stride;
  const uint32_t *rowA = pool + p.env_off[2 * s];
  const uint32_t *rowB = pool + p.env_off[2 * s + 2];
  const int hmin = hA < hB ? hA : hB;
  int32_t M = -kBig;
  for (int r = lane; r < hmin; r += 32) {
    const int32_t ra = (int32_t)(rowA[r] >> 16), lb = (int32_t)(rowB[r] & 0xffffu);
    M = max(M, ra - lb);
  }
  M = warp_max(M);
  int32_t d = wA - M;
  if (d < 0) d = 0;
  const int32_t off = wA - d;
  int a_free = 1, b_free = 1;
  int32_t carry_max = -kBig, carry_min = kBig;  // over rows of A / of B above the chunk
  const int hmax = hA > hB ? hA : hB;
  for (int base = 0; base < hmax; base += 32) {
    const int r = base + lane;
    const int32_t ra = r < hA ? (int32_t)(rowA[r] >> 16) : -kBig;
    const int32_t lb = r < hB ? off + (int32_t)(rowB[r] & 0xffffu) : kBig;
    // exclusive prefix max of R'_A and prefix min of off + L'_B
    const int32_t imax = warp_scan_incl<true>(ra);
    const int32_t imin = warp_scan_incl<false>(lb);
    int32_t emax = __shfl_up_sync(0xffffffffu, imax, 1);
    int32_t emin = __shfl_up_sync(0xffffffffu, imin, 1);
    if (lane == 0) { emax = -kBig; emin = kBig; }
    emax = max(emax, carry_max);
    emin = min(emin, carry_min);
    if (r >= 1 && r < hB && lb < emax) b_free = 0;
    if (r >= 1 && r < hA && ra > emin) a_free = 0;
    carry_max = max(carry_max, __shfl_sync(0xffffffffu, imax, 31));
    carry_min = min(carry_min, __shfl_sync(0xffffffffu, imin, 31));
  }
  a_free = __all_sync(0xffffffffu, a_free);
  b_free = __all_sync(0xffffffffu, b_free);
  if (lane == 0) {
    p.dnext[ps] = d;
    p.pflags[ps] = (uint8_t)((a_free ? 0 : 1) | (b_free ? 0 : 2));
  }
}

}  // namespace

void launch_layout(const Pack &p, cudaStream_t st) { layout_kernel<<<kScales + 1, 1024, 0, st>>>(p); }

void launch_raster(const Pack &p, int j_lo, int j_hi, cudaStream_t st) {
  const int nj = j_hi - j_lo + 1;
  // candidates per warp: enough warps to fill the GPU, as many candidates
  // per warp as that allows (each warp walks its candidates incrementally)
  int64_t G = ((int64_t)nj * p.n + 32767) / 32768;
  G = G < 1 ? 1 : (G > nj ? nj : G);
  const int64_t groups = (nj + G - 1) / G;
  const int64_t warps = (int64_t)p.n * groups;
  const int64_t blocks = (warps * 32 + kRasterThreads - 1) / kRasterThreads;
  raster_kernel<<<(unsigned)blocks, kRasterThreads, 0, st>>>(p, j_lo, nj, (int)G);
}

void launch_hcompact(const Pack &p, int j_lo, int j_hi, cudaStream_t st) {
  const int nj = j_hi - j_lo + 1;
  const int64_t warps = (int64_t)p.n * nj;
  const int64_t blocks = (warps * 32 + 255) / 256;
  hcompact_kernel<<<(unsigned)blocks, 256, 0, st>>>(p, j_lo, nj);
}

}  // namespace tabi
