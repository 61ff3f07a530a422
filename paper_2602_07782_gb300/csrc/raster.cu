// Envelope rasterizer (App. A "Parallel Pushing Algorithm", Sec. 4.1.2, Sec. 5
// gutters).
//
// For each candidate scale k/1024 and sorted chart, one warp produces
//   * per padded column i (w' = w + 2g of them): Top'(i) | Bot'(i) << 16,
//   * per padded row r (h' = h + 2g of them):   L'(r) | R'(r) << 16,
// packed as uint32 into that scale's envelope pool, plus the chart's padded
// size and maximum bottom.  Lane l of chunk t handles raw column 32t + l:
// the local-AABB pieces meeting the open column interval give one bound, the
// OBB's boundary lines (minimum at the box corner if the corner falls inside
// the column, else at the nearer column end) the other; the tighter wins.
// The gutter dilation min/max over raw columns i-2g..i takes the values from
// lanes l-o of the current chunk or, across the chunk seam, of the previous
// chunk (kept in registers), so each raw value is computed exactly once.
//
// The pool layout is fixed by the sizes at k = 1024 (the largest scale), so
// one prefix sum serves every candidate.
#include "tabi_internal.cuh"

namespace tabi {
namespace {

constexpr int32_t kBig = 0x3fffffff;

// Raw bounds of column c (axis = 0) or row c (axis = 1) at scale k.
// Column: lo = TopEdge, hi = BottomEdge.  Row: lo = left, hi = right.
__device__ __forceinline__ void raw_bounds(const ChartShape &sh, int64_t k, int64_t c, int axis,
                                           uint32_t flags, int64_t len_other, int32_t &lo_out,
                                           int32_t &hi_out) {
  const int64_t ext = axis == 0 ? sh.Wq : sh.Hq;  // extent along the scanned axis
  const int64_t a = c * kFix;
  const int64_t b = min((c + 1) * kFix, ext * k);
  int64_t lo = 0, hi = len_other;
  if (flags & TABI_F_LAABB) {
    int64_t pl = 0x7fffffffffffffffLL, ph = -0x7fffffffffffffffLL;
#pragma unroll
    for (int i = 0; i < kSlices; ++i) {
      const int64_t s0 = (int64_t)i * ext / kSlices * k, s1 = (int64_t)(i + 1) * ext / kSlices * k;
      if (s0 < b && s1 > a) {
        const int64_t l = axis == 0 ? sh.tlo[i] : sh.llo[i];
        const int64_t h = axis == 0 ? sh.bhi[i] : sh.rhi[i];
        pl = l < pl ? l : pl;
        ph = h > ph ? h : ph;
      }
    }
    lo = max(lo, floor_fix(pl * k));
    hi = min(hi, ceil_fix(ph * k));
  }
  if ((flags & TABI_F_OBB) && sh.m > 0) {
    const int64_t C = kObbCos[sh.m], S = kObbSin[sh.m];
    const int64_t N = C * C + S * S;
    const int64_t U0 = sh.u0 * k, U1 = sh.u1 * k, V0 = sh.v0 * k, V1 = sh.v1 * k;
    const int64_t aN = a * N, bN = b * N;
    if (axis == 0) {
      // top: y(X) = max((U0 - X C)/S, (V0 + X S)/C); corner u = U0, v = V0
      const int64_t xc = U0 * C - V0 * S;
      int64_t t;
      if (aN <= xc && xc <= bN) {
        t = floor_div(U0 * S + V0 * C, N * kFix);
      } else {
        const int64_t X = xc < aN ? a : b;
        t = max(floor_div(U0 - X * C, S * kFix), floor_div(V0 + X * S, C * kFix));
      }
      // bottom: y(X) = min((U1 - X C)/S, (V1 + X S)/C); corner u = U1, v = V1
      const int64_t xb = U1 * C - V1 * S;
      int64_t bo;
      if (aN <= xb && xb <= bN) {
        bo = ceil_div(U1 * S + V1 * C, N * kFix);
      } else {
        const int64_t X = xb < aN ? a : b;
        bo = min(ceil_div(U1 - X * C, S * kFix), ceil_div(V1 + X * S, C * kFix));
      }
      lo = max(lo, t);
      hi = min(hi, bo);
    } else {
      // left: x(Y) = max((U0 - Y S)/C, (Y C - V1)/S); corner u = U0, v = V1
      const int64_t yl = U0 * S + V1 * C;
      int64_t l;
      if (aN <= yl && yl <= bN) {
        l = floor_div(U0 * C - V1 * S, N * kFix);
      } else {
        const int64_t Y = yl < aN ? a : b;
        l = max(floor_div(U0 - Y * S, C * kFix), floor_div(Y * C - V1, S * kFix));
      }
      // right: x(Y) = min((U1 - Y S)/C, (Y C - V0)/S); corner u = U1, v = V0
      const int64_t yr = U1 * S + V0 * C;
      int64_t r;
      if (aN <= yr && yr <= bN) {
        r = ceil_div(U1 * C - V0 * S, N * kFix);
      } else {
        const int64_t Y = yr < aN ? a : b;
        r = min(ceil_div(U1 - Y * S, C * kFix), ceil_div(Y * C - V0, S * kFix));
      }
      lo = max(lo, l);
      hi = min(hi, r);
    }
  }
  // keep each scanline a non-empty interval inside [0, len_other]
  lo = max((int64_t)0, min(lo, len_other - 1));
  hi = max(lo + 1, min(hi, len_other));
  lo_out = (int32_t)lo;
  hi_out = (int32_t)hi;
}

// One axis of one chart: raw scanlines 0..len-1, padded 0..len+2g-1.
__device__ __forceinline__ int32_t warp_axis(const ChartShape &sh, int64_t k, int axis, int64_t len,
                                             int64_t len_other, int g, uint32_t flags,
                                             uint32_t *__restrict__ dst) {
  const int lane = threadIdx.x & 31;
  const int64_t padded = len + 2 * g;
  int32_t prev_lo = kBig, prev_hi = -kBig;
  int32_t maxhi = 0;
  for (int64_t base = 0; base < padded; base += 32) {
    const int64_t c = base + lane;
    int32_t lo = kBig, hi = -kBig;
    if (c < len) raw_bounds(sh, k, c, axis, flags, len_other, lo, hi);
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

__global__ void __launch_bounds__(256) raster_kernel(Pack p, int j_lo, int nj) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t n = p.n;
  if (gw >= n * nj) return;
  if (*(volatile int32_t *)p.found >= 0) return;  // a larger scale already succeeded
  if (*(volatile uint32_t *)p.err) return;        // invalid input or pool overflow: write nothing
  const int j = j_lo + (int)(gw / n);
  const int s = (int)(gw % n);
  const int64_t k = 16 * (j + 1);
  const ChartShape sh = p.shape[s];
  const int64_t w = (sh.Wq * k + kFix - 1) >> 18, h = (sh.Hq * k + kFix - 1) >> 18;
  const int32_t off = p.env_off[2 * s], wcap = p.env_off[2 * s + 1];
  const int g = p.g;
  uint32_t *base = p.pool + (int64_t)j * p.pool_stride + off;
  const int32_t maxbot = warp_axis(sh, k, 0, w, h, g, p.flags, base);
  warp_axis(sh, k, 1, h, w, g, p.flags, base + wcap);
  if (lane == 0) {
    int32_t *m = p.meta + ((int64_t)j * n + s) * 4;
    m[0] = (int32_t)(w + 2 * g);
    m[1] = (int32_t)(h + 2 * g);
    m[2] = off;
    m[3] = maxbot;
  }
}

// Pool layout from the sizes at k = 1024 (one CTA; exclusive scan).
__global__ void __launch_bounds__(1024) layout_kernel(Pack p) {
  __shared__ int64_t part[32];
  __shared__ int64_t carry;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < p.n; base += 1024) {
    const int s = base + tid;
    int64_t sz = 0, wp = 0;
    if (s < p.n) {
      const ChartShape &sh = p.shape[s];
      wp = ((sh.Wq + 255) >> 8) + 2 * p.g;
      const int64_t hp = ((sh.Hq + 255) >> 8) + 2 * p.g;
      sz = (wp + hp + 3) & ~3LL;  // 16-byte aligned segments
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
      p.env_off[2 * s] = (int32_t)excl;
      p.env_off[2 * s + 1] = (int32_t)wp;
    }
    __syncthreads();
    if (tid == 1023) carry = excl + sz;
    __syncthreads();
  }
  if (tid == 0 && carry > p.pool_cap) atomicOr(p.err, kErrPool);
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
  const uint32_t *pool = p.pool + (int64_t)j * p.pool_stride;
  const uint32_t *rowA = pool + p.env_off[2 * s] + p.env_off[2 * s + 1];
  const uint32_t *rowB = pool + p.env_off[2 * s + 2] + p.env_off[2 * s + 3];
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

void launch_layout(const Pack &p, cudaStream_t st) { layout_kernel<<<1, 1024, 0, st>>>(p); }

void launch_raster(const Pack &p, int j_lo, int j_hi, cudaStream_t st) {
  const int nj = j_hi - j_lo + 1;
  const int64_t warps = (int64_t)p.n * nj;
  const int64_t blocks = (warps * 32 + 255) / 256;
  raster_kernel<<<(unsigned)blocks, 256, 0, st>>>(p, j_lo, nj);
}

void launch_hcompact(const Pack &p, int j_lo, int j_hi, cudaStream_t st) {
  const int nj = j_hi - j_lo + 1;
  const int64_t warps = (int64_t)p.n * nj;
  const int64_t blocks = (warps * 32 + 255) / 256;
  hcompact_kernel<<<(unsigned)blocks, 256, 0, st>>>(p, j_lo, nj);
}

}  // namespace tabi
