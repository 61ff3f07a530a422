// Device routines the rasterizer and the prefix-sum tail share: drawing one
// axis of a chart's envelope, the per-(chart, scale) constants at any scale,
// the compacting distance of a drawn pair, and that distance for two
// charts drawn on the fly.
#pragma once

#include "raster_math.cuh"
#include "tabi_internal.cuh"

namespace tabi {

constexpr int32_t kBig = 0x3fffffff;

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

// Inclusive max / min scan over an aligned group of G lanes.
template <int G, bool kMax>
__device__ __forceinline__ int32_t group_scan_incl(int32_t v, unsigned gm) {
  const int lane = threadIdx.x & (G - 1);
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    const int32_t u = __shfl_up_sync(gm, v, o, G);
    if (lane >= o) v = kMax ? (u > v ? u : v) : (u < v ? u : v);
  }
  return v;
}

// Compacting distance and interlock flags (Sec. 4.1.2, App. A) of the drawn
// pair (s, s+1) of candidate j, by an aligned group of G lanes: A = s left
// of B = s+1, top-aligned:  d = w'_A - max_r (R'_A(r) - L'_B(r));  B may
// move up relative to A iff every row of B stays right of all rows of A
// above it; A may move up relative to B iff every row of A stays left of
// all rows of B above it.
// The pair's sizes and rows (loads only, so a caller can issue them before
// it knows whether it needs them).
struct PairRows {
  int64_t ps;
  int32_t wA, hA, hB;
  const uint32_t *rowA, *rowB;
};
__device__ __forceinline__ PairRows pair_rows(const Pack &p, int at, int j, int s) {
  PairRows r;
  r.ps = (int64_t)j * p.N + s;
  const int32_t *ma = p.meta + r.ps * 4, *mb = ma + 4;
  r.wA = ma[0];
  r.hA = ma[1];
  r.hB = mb[1];
  const uint32_t *pool = p.pool + p.abase[region(at, j, 1)];
  r.rowA = pool + p.rowstart[r.ps];
  r.rowB = pool + p.rowstart[r.ps + 1];
  return r;
}

template <int G>
__device__ __forceinline__ void compact_rows(const Pack &p, const PairRows &pr, int lane, unsigned gm) {
  const int64_t ps = pr.ps;
  const int32_t wA = pr.wA, hA = pr.hA, hB = pr.hB;
  const uint32_t *rowA = pr.rowA, *rowB = pr.rowB;
  const int hmin = hA < hB ? hA : hB;
  int32_t M = -kBig;
  for (int r = lane; r < hmin; r += G) {
    const int32_t ra = (int32_t)(rowA[r] >> 16), lb = (int32_t)(rowB[r] & 0xffffu);
    M = max(M, ra - lb);
  }
  M = group_max<G>(M, gm);
  int32_t d = wA - M;
  if (d < 0) d = 0;
  const int32_t off = wA - d;
  int a_free = 1, b_free = 1;
  int32_t carry_max = -kBig, carry_min = kBig;  // over rows of A / of B above the chunk
  const int hmax = hA > hB ? hA : hB;
  for (int base = 0; base < hmax; base += G) {
    const int r = base + lane;
    const int32_t ra = r < hA ? (int32_t)(rowA[r] >> 16) : -kBig;
    const int32_t lb = r < hB ? off + (int32_t)(rowB[r] & 0xffffu) : kBig;
    // exclusive prefix max of R'_A and prefix min of off + L'_B
    const int32_t imax = group_scan_incl<G, true>(ra, gm);
    const int32_t imin = group_scan_incl<G, false>(lb, gm);
    int32_t emax = __shfl_up_sync(gm, imax, 1, G);
    int32_t emin = __shfl_up_sync(gm, imin, 1, G);
    if (lane == 0) { emax = -kBig; emin = kBig; }
    emax = max(emax, carry_max);
    emin = min(emin, carry_min);
    if (r >= 1 && r < hB && lb < emax) b_free = 0;
    if (r >= 1 && r < hA && ra > emin) a_free = 0;
    carry_max = max(carry_max, __shfl_sync(gm, imax, G - 1, G));
    carry_min = min(carry_min, __shfl_sync(gm, imin, G - 1, G));
  }
  a_free = __all_sync(gm, a_free);
  b_free = __all_sync(gm, b_free);
  if (lane == 0) {
    p.dnext[ps] = d;
    p.pflags[ps] = (uint8_t)((a_free ? 0 : 1) | (b_free ? 0 : 2));
  }
}

template <int G>
__device__ __forceinline__ void compact_pair(const Pack &p, int at, int j, int s, int lane, unsigned gm) {
  compact_rows<G>(p, pair_rows(p, at, j, s), lane, gm);
}

// The constants of one chart at any scale k (1 <= k <= 1024) for one or both
// axes, lane-parallel, into a0 / a1 (the rasterizer walks the candidate grid
// and carries the corners from one candidate to the next instead): lane i
// < 10 the axis-0 piece and cross piece i, lane 10 + i those of axis 1
// (see raster_kernel), lanes 20 and 21 the OBB lines of each axis, lanes
// 24-31 the eight corner quantities, each by one division.  Ends with the
// warp synchronised.
__device__ __forceinline__ void setup_at_k(const Pack &p, const ChartShape &sh, int64_t k, rmath::AxisK *a0,
                                           rmath::AxisK *a1) {
  const int lane = threadIdx.x & 31;
  const bool use_l = (p.flags & TABI_F_LAABB) != 0, use_o = (p.flags & TABI_F_OBB) != 0;
  const int m = sh.m;
  const int64_t C = kObbCos[m], S = kObbSin[m];
  if (lane < 2 * rmath::kK) {
    const int ax = lane >= rmath::kK, i = lane - ax * rmath::kK;
    rmath::AxisK *a = ax ? a1 : a0;
    if (a) {
      const uint32_t ext = (uint32_t)(ax ? sh.Hq : sh.Wq), oth = (uint32_t)(ax ? sh.Wq : sh.Hq);
      const int sl = i * p.laabb_k / rmath::kK;
      rmath::setup_piece(*a, i, i * ext / rmath::kK, (i + 1) * ext / rmath::kK, (uint32_t)k,
                         (uint32_t)(ax ? sh.xlo[i] : sh.ylo[i]), (uint32_t)(ax ? sh.xhi[i] : sh.yhi[i]));
      rmath::setup_cross(*a, i, (uint32_t)(ax ? sh.ylo[i] : sh.xlo[i]), (uint32_t)(ax ? sh.yhi[i] : sh.xhi[i]), ext,
                         (uint32_t)k, (uint32_t)(sl * rmath::kK / p.laabb_k) * oth / rmath::kK,
                         (uint32_t)((sl + 1) * rmath::kK / p.laabb_k) * oth / rmath::kK);
    }
  } else if (lane < 2 * rmath::kK + 2) {
    const int ax = lane - 2 * rmath::kK;
    rmath::AxisK *a = ax ? a1 : a0;
    if (a) {
      rmath::setup_obb_fixed(*a, ax, m, C, S, kObbDivCos[m], kObbDivSin[m], use_l, use_o);
      rmath::setup_obb_k(*a, ax, sh.Wq, sh.Hq, k, C, S, sh.u0, sh.u1, sh.v0, sh.v1);
    }
  } else if (lane >= 24 && use_o && m > 0) {
    const int item = lane - 24, ax = item >> 2;
    rmath::AxisK *a = ax ? a1 : a0;
    if (a) {
      rmath::CornerQ cq;
      rmath::corner_at(cq, item, k, C, S, sh.u0, sh.u1, sh.v0, sh.v1);
      rmath::corner_store(cq, item, *a, (ax ? sh.Hq : sh.Wq) * k);
    }
  }
  __syncwarp();
}

// max_r (R'_A(r) - L'_B(r)) over the padded rows both charts have, drawn on
// the fly from the row constants (axis 1) of A and B, by a warp: lane l of
// chunk t takes padded row 32 t + l; the gutter dilation takes the raw
// values of the rows before it from the lanes below or, across the chunk
// seam, from the previous chunk (as warp_axis).
__device__ __forceinline__ int32_t warp_pair_reach(const rmath::AxisK &A, const rmath::AxisK &B, int g) {
  const int lane = threadIdx.x & 31;
  const int32_t hmin = min(A.len, B.len) + 2 * g;
  int32_t prev_hi = -kBig, prev_lo = kBig, M = -kBig;
  for (int32_t base = 0; base < hmin; base += 32) {
    const int32_t c = base + lane;
    int32_t alo, ahi = -kBig, blo = kBig, bhi;
    if (c < A.len) rmath::scanline(A, c, alo, ahi);
    if (c < B.len) rmath::scanline(B, c, blo, bhi);
    int32_t dhi = ahi, dlo = blo;
    for (int o = 1; o <= 2 * g; ++o) {
      const int32_t ch = __shfl_sync(0xffffffffu, ahi, (lane - o) & 31);
      const int32_t ph = __shfl_sync(0xffffffffu, prev_hi, (lane - o) & 31);
      const int32_t cl = __shfl_sync(0xffffffffu, blo, (lane - o) & 31);
      const int32_t pl = __shfl_sync(0xffffffffu, prev_lo, (lane - o) & 31);
      dhi = max(dhi, lane >= o ? ch : ph);
      dlo = min(dlo, lane >= o ? cl : pl);
    }
    if (c < hmin) M = max(M, dhi + 2 * g - dlo);
    prev_hi = ahi;
    prev_lo = blo;
  }
  return warp_max(M);
}

// The row constants (axis 1) of one chart at any scale k by an aligned
// group of G >= 8 lanes (glane: the lane within the group): the pieces and
// cross pieces spread over the lanes, the OBB lines on lane 0, the four row
// corners on lanes 4-7.  The caller synchronises the group after.
template <int G>
__device__ __forceinline__ void group_setup_rows(const Pack &p, const ChartShape &sh, int64_t k, rmath::AxisK &a,
                                                 int glane) {
  const bool use_l = (p.flags & TABI_F_LAABB) != 0, use_o = (p.flags & TABI_F_OBB) != 0;
  const int m = sh.m;
  const int64_t C = kObbCos[m], S = kObbSin[m];
  const uint32_t ext = (uint32_t)sh.Hq, oth = (uint32_t)sh.Wq;
  for (int i = glane; i < rmath::kK; i += G) {
    const int sl = i * p.laabb_k / rmath::kK;
    rmath::setup_piece(a, i, i * ext / rmath::kK, (i + 1) * ext / rmath::kK, (uint32_t)k, (uint32_t)sh.xlo[i],
                       (uint32_t)sh.xhi[i]);
    rmath::setup_cross(a, i, (uint32_t)sh.ylo[i], (uint32_t)sh.yhi[i], ext, (uint32_t)k,
                       (uint32_t)(sl * rmath::kK / p.laabb_k) * oth / rmath::kK,
                       (uint32_t)((sl + 1) * rmath::kK / p.laabb_k) * oth / rmath::kK);
  }
  if (glane == 0) {
    rmath::setup_obb_fixed(a, 1, m, C, S, kObbDivCos[m], kObbDivSin[m], use_l, use_o);
    rmath::setup_obb_k(a, 1, sh.Wq, sh.Hq, k, C, S, sh.u0, sh.u1, sh.v0, sh.v1);
  } else if (glane >= 4 && glane < 8 && use_o && m > 0) {
    rmath::CornerQ cq;
    rmath::corner_at(cq, glane, k, C, S, sh.u0, sh.u1, sh.v0, sh.v1);  // items 4-7: the row corners
    rmath::corner_store(cq, glane, a, sh.Hq * k);
  }
}

// warp_pair_reach by an aligned group of G lanes (2g < G: the gutter
// dilation reaches back one chunk at most).
template <int G>
__device__ __forceinline__ int32_t group_pair_reach(const rmath::AxisK &A, const rmath::AxisK &B, int g, int glane,
                                                    unsigned gm) {
  const int32_t hmin = min(A.len, B.len) + 2 * g;
  int32_t prev_hi = -kBig, prev_lo = kBig, M = -kBig;
  for (int32_t base = 0; base < hmin; base += G) {
    const int32_t c = base + glane;
    int32_t alo, ahi = -kBig, blo = kBig, bhi;
    if (c < A.len) rmath::scanline(A, c, alo, ahi);
    if (c < B.len) rmath::scanline(B, c, blo, bhi);
    int32_t dhi = ahi, dlo = blo;
    for (int o = 1; o <= 2 * g; ++o) {
      const int src = (glane - o) & (G - 1);
      const int32_t ch = __shfl_sync(gm, ahi, src, G), ph = __shfl_sync(gm, prev_hi, src, G);
      const int32_t cl = __shfl_sync(gm, blo, src, G), pl = __shfl_sync(gm, prev_lo, src, G);
      dhi = max(dhi, glane >= o ? ch : ph);
      dlo = min(dlo, glane >= o ? cl : pl);
    }
    if (c < hmin) M = max(M, dhi + 2 * g - dlo);
    prev_hi = ahi;
    prev_lo = blo;
  }
  return group_max<G>(M, gm);
}

}  // namespace tabi
