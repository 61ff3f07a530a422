// Chart preparation (Sec. 3.1, Sec. 4.1.1, App. A) and the height sort.
//
// prep_kernel: a group of G lanes per chart (G = 32, 16, 8 or 4, chosen by
// the batch's chart count: narrow groups keep more charts in flight -- the
// kernel is bound by latency, not issue -- once there are enough of them).  Lanes stride over the chart's edges; the per-slice
// extrema and the per-angle OBB extents are combined with shuffles inside
// the group (its own lane mask), so no atomics are needed.  Three slice passes mirror the
// orientation logic: slices of the rotated chart decide the vertical
// reflection, slices of the vertically reflected chart decide the horizontal
// one, slices of the final chart are the local-AABB proxy.  A reflection
// mirrors the other axis' slice extents exactly, so only the slices along
// the reflected axis are recomputed (two or three slab passes, not five).
//
// sort_kernel: one CTA per atlas, stable LSD radix sort (three 7-bit digits of
// 2^21 - 1 - Hq), so charts come out by decreasing AABB height with ties in
// input order.  Ranking inside a warp uses __match_any_sync.
#include "tabi_internal.cuh"

namespace tabi {
namespace {

constexpr int64_t kI64Max = 0x7fffffffffffffffLL;
constexpr int64_t kI64Min = -kI64Max - 1;

// Chart-local transform: translate the AABB min to the origin, rotate
// (x, y) -> (y, W0 - x) when wider than tall, then the reflections.  Input
// coordinates lie in (-2^20, 2^20), so every intermediate is in [0, 2^21]
// and 32-bit arithmetic is exact.
struct Xf {
  int32_t minx, miny, W0, Wq, Hq;
  int rot, fy, fx;
  __device__ __forceinline__ void apply(int32_t vx, int32_t vy, int32_t &x, int32_t &y) const {
    const int32_t tx = vx - minx, ty = vy - miny;
    if (rot) { x = ty; y = W0 - tx; } else { x = tx; y = ty; }
    if (fy) y = Hq - y;
    if (fx) x = Wq - x;
  }
};

// floor and ceil of num / d for d > 0 whose quotient is known to lie in
// [-2^21, 2^21] (|num| < 2^43): a float estimate of the quotient is within
// one of the floor (relative error below 2^-22), and the exact integer
// remainder corrects it.
__device__ __forceinline__ void floor_ceil_div(int64_t num, int32_t d, int32_t &f, int32_t &c) {
  int32_t q = (int32_t)floorf((float)num * (1.0f / (float)d));
  int64_t r = num - (int64_t)q * d;
  if (r < 0) { --q; r += d; }
  else if (r >= d) { ++q; r -= d; }
  f = q;
  c = q + (r != 0);
}

// Local AABBs of the K slices along one axis: for slice i = [B_i, B_{i+1}]
// (B_i = floor(i * ext / K), closed), floor(min) and ceil(max) of the other
// coordinate over the polygon's boundary inside the slab.  That part of the
// boundary is spanned by the vertices inside the slab and the points where
// edges cross its bounding lines, so each lane takes its vertices (exact
// values) and its edges' crossings of the inner lines B_1 .. B_{K-1}
// strictly between the edge's ends (a crossing of B_m belongs to slices
// m-1 and m).  K is 10 (App. A) or 2 or 5 (the Tab. 13 ablation).
// Coordinates of the normalised chart lie in [0, 2^21], so everything but
// the crossing numerators fits 32 bits.  Every lane of the group ends with
// all values.
template <int G, int K>
__device__ void group_slices(const int32_t *__restrict__ v, int nv, const Xf &xf, bool xaxis,
                             int64_t ext, int32_t (&lo)[K], int32_t (&hi)[K]) {
  const int lane = threadIdx.x & (G - 1);
  const unsigned gm = group_mask<G>();
  int32_t B[K + 1];
#pragma unroll
  for (int i = 0; i <= K; ++i) B[i] = (int32_t)((int64_t)i * ext / K);
#pragma unroll
  for (int i = 0; i < K; ++i) { lo[i] = 0x7fffffff; hi[i] = -0x7fffffff - 1; }
  for (int e = lane; e < nv; e += G) {
    const int e1 = (e + 1 == nv) ? 0 : e + 1;
    int32_t x0, y0, x1, y1;
    xf.apply(v[2 * e], v[2 * e + 1], x0, y0);
    xf.apply(v[2 * e1], v[2 * e1 + 1], x1, y1);
    const int32_t u0 = xaxis ? x0 : y0, w0 = xaxis ? y0 : x0;
    const int32_t u1 = xaxis ? x1 : y1, w1 = xaxis ? y1 : x1;
    // vertex e, in every slice that contains it
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (B[i] <= u0 && u0 <= B[i + 1]) { lo[i] = min(lo[i], w0); hi[i] = max(hi[i], w0); }
    // crossings of edge (e, e+1) with the inner slab lines
    const int32_t ul = min(u0, u1), ur = max(u0, u1);
    unsigned mask = 0;
#pragma unroll
    for (int m = 1; m < K; ++m)
      if (ul < B[m] && B[m] < ur) mask |= 1u << m;
    if (mask) {
      const int32_t sgn = u1 > u0 ? 1 : -1;
      const int32_t d = (u1 - u0) * sgn;
      while (mask) {
        const int m = __ffs(mask) - 1;
        mask &= mask - 1;
        const int32_t Bm = (int32_t)((int64_t)m * ext / K);
        const int64_t num = sgn * ((int64_t)w0 * (u1 - u0) + (int64_t)(Bm - u0) * (w1 - w0));
        int32_t f, c;
        floor_ceil_div(num, d, f, c);
#pragma unroll
        for (int i = 0; i < K; ++i)
          if (i == m - 1 || i == m) { lo[i] = min(lo[i], f); hi[i] = max(hi[i], c); }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < K; ++i) {
    lo[i] = group_min<G>(lo[i], gm);
    hi[i] = group_max<G>(hi[i], gm);
  }
}

// One chart (global input index c) of the batch, by a group of G lanes,
// with K local AABBs per axis, K dividing 10.  The records keep ten slots
// per axis: slot t holds slice floor(t K / 10).  Slice s of K spans the
// ten-slice boundaries floor(i E / 10) for i = 10 s / K .. 10 (s + 1) / K
// (floor(s E / K) = floor((10 s / K) E / 10)), so its slots' open intervals
// tile its own and an envelope over the ten slots equals one over the K
// slices: the rasterizer needs no count.
template <int G, int K>
__device__ __forceinline__ void prep_chart(const Pack &p, int c) {
  const int lane = threadIdx.x & (G - 1);
  const unsigned gm = group_mask<G>();
  const int at = p.catl[c];
  const AtlasDesc &ad = p.atl[at];
  const int lc = c - ad.cb;  // index within its atlas
  const uint32_t a = ad.offsets[lc], b = ad.offsets[lc + 1];
  const int nv = (int)(b - a);
  const int32_t *v = ad.verts + 2 * (size_t)a;
  tabi_chart_info *inf = p.info + c;
  ChartShape *sh = p.shape_in + c;

  // Sec. 3.1: the chart's AABB (and input validation)
  int32_t mnx = 0x7fffffff, mny = 0x7fffffff, mxx = -0x7fffffff - 1, mxy = -0x7fffffff - 1;
  int bad = (b < a) || (nv < 3) || (b > (uint32_t)ad.nv);
  if (!bad) {
    for (int i = lane; i < nv; i += G) {
      const int32_t x = v[2 * i], y = v[2 * i + 1];
      bad |= (x <= -(1 << 20)) | (x >= (1 << 20)) | (y <= -(1 << 20)) | (y >= (1 << 20));
      mnx = min(mnx, x); mxx = max(mxx, x);
      mny = min(mny, y); mxy = max(mxy, y);
    }
  }
  bad = __any_sync(gm, bad);
  mnx = group_min<G>(mnx, gm); mxx = group_max<G>(mxx, gm);
  mny = group_min<G>(mny, gm); mxy = group_max<G>(mxy, gm);
  const int64_t W0 = (int64_t)mxx - mnx, H0 = (int64_t)mxy - mny;
  const int rot = W0 > H0;  // rotate to be taller than wide (strictly wider)
  const int64_t Wq = rot ? H0 : W0, Hq = rot ? W0 : H0;
  if (bad || Wq < 256 || Hq < 256) {
    // rejected: keep a harmless one-texel box so later kernels stay in bounds
    if (lane == 0) {
      inf->orig = lc; inf->valid = 0; inf->Wq = 0; inf->Hq = 0;
      p.carea[c] = 0;
      p.barea[c] = 0;
      sh->Wq = 256; sh->Hq = 256; sh->m = 0; sh->pad = 0;
      sh->u0 = sh->u1 = sh->v0 = sh->v1 = 0;
      atomicOr(p.err + at, kErrInvalid);
    }
    for (int i = lane; i < kSlices; i += G) {
      sh->ylo[i] = 0; sh->yhi[i] = 256; sh->xlo[i] = 0; sh->xhi[i] = 256;
    }
    return;
  }
  Xf xf{mnx, mny, (int32_t)W0, (int32_t)Wq, (int32_t)Hq, rot, 0, 0};

  // Twice the polygon's area (shoelace, input coordinates).  The area
  // bound on the candidate scales needs the area a chart surely covers,
  // which |shoelace| / 2 is for a simple polygon but not for a loop that
  // winds twice or crosses itself (its shoelace can exceed its cover).  So
  // the bound takes a chart's area only where one pass certifies the loop
  // simple: every edge turns strictly the same way around the point
  // c = floor(vertex mean) (cross(v_i - c, v_i+1 - c) all > 0 or all < 0)
  // and the loop winds around c exactly once -- then every ray from c meets
  // the loop once, so it is a simple polygon, star-shaped about c.  Other
  // loops (non-star simple polygons among them) enter the bound with area
  // 0, which keeps it a valid lower bound; only its strength changes.
  {
    int64_t a2 = 0, sx = 0, sy = 0;
    for (int e = lane; e < nv; e += G) {
      const int e1 = (e + 1 == nv) ? 0 : e + 1;
      a2 += (int64_t)v[2 * e] * v[2 * e1 + 1] - (int64_t)v[2 * e1] * v[2 * e + 1];
      sx += v[2 * e];
      sy += v[2 * e + 1];
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      a2 += __shfl_xor_sync(gm, a2, o);
      sx += __shfl_xor_sync(gm, sx, o);
      sy += __shfl_xor_sync(gm, sy, o);
    }
    // floor of the vertex mean (|sum| < 2^38); offsets from it below 2^21
    const int64_t cx = sx >= 0 ? sx / nv : -((-sx + nv - 1) / nv);
    const int64_t cy = sy >= 0 ? sy / nv : -((-sy + nv - 1) / nv);
    int pos = 1, neg = 1, wn = 0;
    for (int e = lane; e < nv; e += G) {
      const int e1 = (e + 1 == nv) ? 0 : e + 1;
      const int64_t ax = v[2 * e] - cx, ay = v[2 * e + 1] - cy;
      const int64_t bx = v[2 * e1] - cx, by = v[2 * e1 + 1] - cy;
      const int64_t cr = ax * by - bx * ay;  // below 2^43 in size
      pos &= cr > 0;
      neg &= cr < 0;
      // winding number of the loop about c (crossings of the ray y = 0,
      // x > 0, counted with their direction; half-open in y)
      if (ay <= 0) { if (by > 0 && cr > 0) ++wn; }
      else if (by <= 0 && cr < 0) --wn;
    }
    pos = __all_sync(gm, pos);
    neg = __all_sync(gm, neg);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) wn += __shfl_xor_sync(gm, wn, o);
    const unsigned long long aa = (unsigned long long)(a2 < 0 ? -a2 : a2);
    const bool simple = (pos || neg) && (wn == 1 || wn == -1);
    if (lane == 0) {
      p.carea[c] = aa;
      p.barea[c] = simple ? aa : 0ull;
      atomicAdd(p.area2 + at, simple ? aa : 0ull);
      atomicAdd(p.ext_sum + at, (unsigned long long)Hq);  // Hq >= Wq after the rotation
    }
  }
  int32_t ylo[K], yhi[K], xlo[K], xhi[K];

  // App. A chart orientation, vertical reflection: top vs bottom empty area
  group_slices<G, K>(v, nv, xf, true, Wq, ylo, yhi);
  int64_t top = 0, bottom = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int64_t wi = (int64_t)(i + 1) * Wq / K - (int64_t)i * Wq / K;
    top += wi * ylo[i];
    bottom += wi * (Hq - yhi[i]);
  }
  xf.fy = top > bottom;

  // A reflection mirrors the extents of the slices along the other axis
  // exactly (floor(min(H - v)) = H - ceil(max v)); the slices along the
  // reflected axis must be recomputed, their boundaries do not mirror.
  if (xf.fy) {
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const int32_t lo = (int32_t)Hq - yhi[i], hi = (int32_t)Hq - ylo[i];
      ylo[i] = lo;
      yhi[i] = hi;
    }
  }

  // horizontal reflection: left vs right empty area, else bottom-left vs
  // bottom-right of the midline (doubled coordinates)
  group_slices<G, K>(v, nv, xf, false, Hq, xlo, xhi);
  int64_t left = 0, right = 0, bl2 = 0, br2 = 0;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int64_t hj = (int64_t)(j + 1) * Hq / K - (int64_t)j * Hq / K;
    left += hj * xlo[j];
    right += hj * (Wq - xhi[j]);
  }
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int64_t e = Hq - yhi[i];
    const int64_t a2 = 2 * ((int64_t)i * Wq / K), b2 = 2 * ((int64_t)(i + 1) * Wq / K);
    const int64_t lenL = max((int64_t)0, min(b2, Wq) - max(a2, (int64_t)0));
    const int64_t lenR = max((int64_t)0, min(b2, 2 * Wq) - max(a2, Wq));
    bl2 += e * lenL;
    br2 += e * lenR;
  }
  const int64_t diff = left - right;
  const int64_t adiff = diff < 0 ? -diff : diff;
  if (100 * adiff > (int64_t)p.lr_sig * Wq * Hq) xf.fx = diff > 0;
  else xf.fx = bl2 > br2;

  // final local AABBs
  if (xf.fx) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int32_t lo = (int32_t)Wq - xhi[j], hi = (int32_t)Wq - xlo[j];
      xlo[j] = lo;
      xhi[j] = hi;
    }
    group_slices<G, K>(v, nv, xf, true, Wq, ylo, yhi);
  }

  // the final slices into the shape record (ten slots per axis, slot t
  // holding slice t K / 10); Sec. 4.1.1's merge of the two sets happens per
  // scanline in the rasterizer
  for (int t = lane; t < 2 * kSlices; t += G) {
    const int ax = t >= kSlices, i = (t - ax * kSlices) * K / kSlices;
    int32_t lo = 0, hi = 0;
#pragma unroll
    for (int q = 0; q < K; ++q)
      if (q == i) { lo = ax ? xlo[q] : ylo[q]; hi = ax ? xhi[q] : yhi[q]; }
    if (ax) { sh->xlo[t - kSlices] = lo; sh->xhi[t - kSlices] = hi; }
    else { sh->ylo[t] = lo; sh->yhi[t] = hi; }
  }

  // App. A OBB: 8 angles, extents of u = xC + yS, v = -xS + yC.  Lane l
  // takes angle l % 8 over every (G/8)-th vertex from l / 8; the lanes of
  // an angle combine by exchanges; then every lane picks the angle of least
  // area / (C^2 + S^2) in angle order, exactly as a sequential scan over m
  // would (ties to the smaller m).
  int64_t bu0 = 0, bu1 = 0, bv0 = 0, bv1 = 0;
  int best = 0;
  {
    // groups narrower than 8 lanes: lane l takes angles l, l + G, ...
    constexpr int R = G >= 8 ? 1 : 8 / G;
    int64_t u0[R], u1[R], v0[R], v1[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int am = (lane & 7) + G * r;
      const int32_t C = kObbCos[am], S = kObbSin[am];
      u0[r] = kI64Max; u1[r] = kI64Min; v0[r] = kI64Max; v1[r] = kI64Min;
      for (int i = G >= 8 ? lane >> 3 : 0; i < nv; i += G >= 8 ? G / 8 : 1) {
        int32_t x, y;
        xf.apply(v[2 * i], v[2 * i + 1], x, y);
        // |x|, |y| <= 2^21 and C, S <= 2^14: 32 x 32 -> 64-bit products
        const int64_t uu = (int64_t)x * C + (int64_t)y * S, vv = (int64_t)y * C - (int64_t)x * S;
        u0[r] = min(u0[r], uu); u1[r] = max(u1[r], uu);
        v0[r] = min(v0[r], vv); v1[r] = max(v1[r], vv);
      }
#pragma unroll
      for (int o = 8; o < G; o <<= 1) {
        u0[r] = min(u0[r], (int64_t)__shfl_xor_sync(gm, u0[r], o));
        u1[r] = max(u1[r], (int64_t)__shfl_xor_sync(gm, u1[r], o));
        v0[r] = min(v0[r], (int64_t)__shfl_xor_sync(gm, v0[r], o));
        v1[r] = max(v1[r], (int64_t)__shfl_xor_sync(gm, v1[r], o));
      }
    }
    __int128 best_area = 0, best_n = 1;
#pragma unroll
    for (int m = 0; m < kAngles; ++m) {
      const int r = m / G < R ? m / G : 0;  // angle m: lane m % G, slot m / G
      const int64_t dum = __shfl_sync(gm, u1[r] - u0[r], m % G, G);
      const int64_t dvm = __shfl_sync(gm, v1[r] - v0[r], m % G, G);
      const int64_t Cm = kObbCos[m], Sm = kObbSin[m];
      const __int128 area = (__int128)dum * dvm;
      const __int128 nrm = (__int128)(Cm * Cm + Sm * Sm);
      if (m == 0 || area * best_n < best_area * nrm) {
        best = m; best_area = area; best_n = nrm;
      }
    }
    int64_t su0 = u0[0], su1 = u1[0], sv0 = v0[0], sv1 = v1[0];
#pragma unroll
    for (int r = 1; r < R; ++r)
      if (best / G == r) { su0 = u0[r]; su1 = u1[r]; sv0 = v0[r]; sv1 = v1[r]; }
    bu0 = __shfl_sync(gm, su0, best % G, G);
    bu1 = __shfl_sync(gm, su1, best % G, G);
    bv0 = __shfl_sync(gm, sv0, best % G, G);
    bv1 = __shfl_sync(gm, sv1, best % G, G);
  }

  // write the records
  if (lane == 0) {
    inf->orig = lc; inf->Wq = (int32_t)Wq; inf->Hq = (int32_t)Hq;
    inf->rot90 = rot; inf->flip_y = xf.fy; inf->flip_x = xf.fx; inf->obb_m = best; inf->valid = 1;
    inf->u0 = bu0; inf->u1 = bu1; inf->v0 = bv0; inf->v1 = bv1;
    inf->area_top = top; inf->area_bot = bottom; inf->area_left = left; inf->area_right = right;
    inf->area_bl2 = bl2; inf->area_br2 = br2;
#pragma unroll
    for (int i = 0; i < kSlices; ++i) {
      const int q = i * K / kSlices;
      inf->ylo[i] = (int32_t)ylo[q]; inf->yhi[i] = (int32_t)yhi[q];
      inf->xlo[i] = (int32_t)xlo[q]; inf->xhi[i] = (int32_t)xhi[q];
    }
    sh->Wq = (int32_t)Wq; sh->Hq = (int32_t)Hq; sh->m = best; sh->pad = 0;
    sh->u0 = bu0; sh->u1 = bu1; sh->v0 = bv0; sh->v1 = bv1;
  }
}

// One group of G lanes per chart.  Groups narrower than a warp run loops
// as long as their chart's vertex count, so a CTA takes tiles of charts and
// orders each tile by vertex count (a counting sort in shared memory)
// before its groups take them: the charts of one warp then have similar
// loop lengths.  The order does not matter otherwise (charts are
// independent).
constexpr int kPrepThreads = 256, kPrepTile = 512, kPrepKeys = 128;
template <int G, int K>
__global__ void __launch_bounds__(kPrepThreads, 2) prep_kernel(const Pack *__restrict__ pp) {
  const Pack &p = *pp;
  if constexpr (G == 32) {
    const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / G;
    for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G; c < p.N; c += groups)
      prep_chart<G, K>(p, (int)c);
  } else {
    __shared__ int32_t order[kPrepTile];
    __shared__ uint8_t key[kPrepTile];
    __shared__ int32_t cnt[kPrepKeys];
    constexpr int kGroups = kPrepThreads / G;
    const int tid = threadIdx.x;
    for (int64_t base = (int64_t)blockIdx.x * kPrepTile; base < p.N; base += (int64_t)gridDim.x * kPrepTile) {
      const int m = (int)min((int64_t)kPrepTile, p.N - base);
      for (int i = tid; i < kPrepKeys; i += kPrepThreads) cnt[i] = 0;
      __syncthreads();
      for (int i = tid; i < m; i += kPrepThreads) {
        const int c = (int)(base + i);
        const AtlasDesc &ad = p.atl[p.catl[c]];
        const int lc = c - ad.cb;
        const int64_t nv = (int64_t)ad.offsets[lc + 1] - ad.offsets[lc];  // checked in prep_chart
        const int k = nv < 0 ? 0 : (nv >= kPrepKeys ? kPrepKeys - 1 : (int)nv);
        key[i] = (uint8_t)k;
        atomicAdd(&cnt[k], 1);
      }
      __syncthreads();
      if (tid < 32) {  // exclusive scan of the key counts (four per lane)
        int v[4], sum = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) { v[r] = cnt[4 * tid + r]; sum += v[r]; }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int u = __shfl_up_sync(0xffffffffu, incl, o);
          if (tid >= o) incl += u;
        }
        int run = incl - sum;
#pragma unroll
        for (int r = 0; r < 4; ++r) { cnt[4 * tid + r] = run; run += v[r]; }
      }
      __syncthreads();
      for (int i = tid; i < m; i += kPrepThreads) order[atomicAdd(&cnt[key[i]], 1)] = (int)(base + i);
      __syncthreads();
      for (int i = tid / G; i < m; i += kGroups) prep_chart<G, K>(p, order[i]);
      __syncthreads();  // the tile's arrays are refilled next
    }
  }
}

// ---------------------------------------------------------------------------
// stable radix sort by decreasing Hq (one CTA)
// ---------------------------------------------------------------------------
constexpr int kSortThreads = kRadixThreads;

// Exclusive scan of three counters over the threads of a CTA (kSortThreads
// threads, in thread order); every thread also gets the totals.
__device__ __forceinline__ void block_scan3(unsigned long long (&v)[3], unsigned long long (&tot)[3]) {
  __shared__ unsigned long long part[3][kSortThreads / 32 + 1];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  unsigned long long inc[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    inc[q] = v[q];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(0xffffffffu, inc[q], o);
      if (lane >= o) inc[q] += u;
    }
    if (lane == 31) part[q][w] = inc[q];
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const unsigned long long x = part[q][lane];
      unsigned long long y = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += u;
      }
      part[q][lane] = y - x;
      if (lane == 31) part[q][32] = y;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    v[q] = part[q][w] + inc[q] - v[q];
    tot[q] = part[q][32];
  }
  __syncthreads();
}

__device__ void sort_atlas(const Pack &p, int at) {
  const int cb = p.atl[at].cb;
  const int n = p.atl[at].n, tid = threadIdx.x;
  uint32_t *kA = p.sort_tmp + 4 * (int64_t)cb, *vA = kA + n, *kB = vA + n, *vB = kB + n;
  for (int c = tid; c < n; c += kSortThreads) {
    kA[c] = (uint32_t)((1 << 21) - 1 - p.shape_in[cb + c].Hq);
    vA[c] = (uint32_t)c;
  }
  radix_sort21(kA, vA, kB, vB, n);  // sorted values in vB, keys in kB
  // the permutation, the sorted heights, and per sorted position the areas
  // and heights of the charts before it (exclusive prefix sums: the area
  // bounds take the certified areas and heights, Sec. 4.4's choice the
  // areas); each thread sums a run of consecutive positions, then a scan
  const int P = (n + kSortThreads - 1) / kSortThreads;
  const int s0 = min(n, tid * P), s1 = min(n, s0 + P);
  unsigned long long v[3] = {0, 0, 0}, tot[3];
  for (int s = s0; s < s1; ++s) {
    const int c = cb + (int32_t)vB[s];
    const int32_t hq = (1 << 21) - 1 - (int32_t)kB[s];
    p.perm[cb + s] = c;
    p.hq[cb + s] = hq;
    v[0] += p.barea[c];
    v[1] += (unsigned long long)hq;
    v[2] += p.carea[c];
  }
  block_scan3(v, tot);
  for (int s = s0; s < s1; ++s) {
    const int c = cb + (int32_t)vB[s];
    p.pre2[cb + s] = v[0];
    p.preE[cb + s] = v[1];
    p.prea[cb + s] = v[2];
    v[0] += p.barea[c];
    v[1] += (unsigned long long)((1 << 21) - 1 - (int32_t)kB[s]);
    v[2] += p.carea[c];
  }
  __syncthreads();
  if (tid == 0) {
    p.area_tot[at] = tot[2];
    // Area bound: placed charts' covers, each dilated by the gutter g, are
    // disjoint and lie in the padded atlas (W + 2g) x (H + 2g).  A connected
    // polygon of area A and larger extent E dilated by g covers at least
    // A + 2 g E + 4 g^2 (every line across it gains 2g); A is taken only
    // for loops certified simple (else 0, see prep_chart).  At scale k/1024 the
    // area is area2 k^2 / 2^37 and the extent E k / 2^18 texels (area2 =
    // twice the area in Q.8^2, E in Q.8), so candidate k can succeed only if
    //   area2 k^2 + 2g 2^19 k sum(E) + 4 g^2 2^37 n <= (W + 2g)(H + 2g) 2^37.
    // Where the prefix-sum tail may apply (Sec. 4.4) its charts may end at
    // the tail's scale, at least k - 14: the charts surely folded row by
    // row at k (head_prefix) count at k, the others at k - 14.  Larger
    // candidates are skipped.
    int jt = kScales - 1;
    if (!(p.flags & TABI_F_EVAL_ALL)) {
      const uint64_t g = (uint64_t)p.g;
      const unsigned __int128 lim =
          (unsigned __int128)(((uint64_t)p.atl[at].W + 2 * g) * ((uint64_t)p.atl[at].H + 2 * g)) << 37;
      const unsigned __int128 fixed = (unsigned __int128)(4 * g * g * (uint64_t)n) << 37;
      const bool hybrid = p.topt > 0 && n > p.hyb_min;
      jt = -1;
      for (int j = 0; j < kScales; ++j) {
        const uint64_t k = 16 * (uint64_t)(j + 1), kr = hybrid ? k - kTailSteps : k;
        const int hp = head_prefix(p.hq + cb, n, (int64_t)k, p.topt, p.atl[at].H, hybrid);
        const unsigned __int128 s2 = hp < n ? p.pre2[cb + hp] : p.area2[at];
        const unsigned __int128 ex = hp < n ? p.preE[cb + hp] : p.ext_sum[at];
        const unsigned __int128 s2r = p.area2[at] - s2, exr = p.ext_sum[at] - ex;
        const unsigned __int128 need = s2 * (k * k) + s2r * (kr * kr) + (((ex * k + exr * kr) * (2 * g)) << 19) + fixed;
        if (need <= lim) jt = j;
      }
    }
    p.jtop[at] = jt;
  }
  __syncthreads();  // the shared histogram is reused by the next atlas
}

// one CTA per atlas (grid-stride over the batch's atlases)
__global__ void __launch_bounds__(kSortThreads) sort_kernel(const Pack *__restrict__ pp) {
  const Pack &p = *pp;
  for (int at = blockIdx.x; at < p.A; at += gridDim.x) sort_atlas(p, at);
}

__global__ void gather_kernel(const Pack *__restrict__ pp) {
  const Pack &p = *pp;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < p.N; s += (int64_t)gridDim.x * blockDim.x) {
    const int c = p.perm[s];
    const ChartShape &sh = p.shape_in[c];
    p.shape[s] = sh;
    p.hq[s] = sh.Hq;
    p.wq[s] = sh.Wq;
  }
}

}  // namespace

template <int K>
void launch_prep_k(const Pack *dp, const Launch &L, cudaStream_t st) {
  switch (L.prep_group) {
    case 32: prep_kernel<32, K><<<L.sms * 8, kPrepThreads, 0, st>>>(dp); break;
    case 16: prep_kernel<16, K><<<L.sms * 8, kPrepThreads, 0, st>>>(dp); break;
    case 8: prep_kernel<8, K><<<L.sms * 8, kPrepThreads, 0, st>>>(dp); break;
    default: prep_kernel<4, K><<<L.sms * 8, kPrepThreads, 0, st>>>(dp); break;
  }
}

void launch_prep(const Pack *dp, const Launch &L, cudaStream_t st) {
  switch (L.laabb_k) {
    case 2: launch_prep_k<2>(dp, L, st); break;
    case 5: launch_prep_k<5>(dp, L, st); break;
    default: launch_prep_k<kSlices>(dp, L, st); break;
  }
}

// Lanes per chart: wide groups while the charts leave the multiprocessors'
// resident warps (two 256-thread CTAs each) idle -- the latency of one
// chart is the prep time then -- narrow ones once they are all busy.
int prep_group_for(int64_t charts, int sms) {
  const int64_t warps = (int64_t)sms * 16;
  return charts <= warps ? 32 : charts <= 2 * warps ? 16 : charts <= 4 * warps ? 8 : 4;
}

void launch_sort(const Pack *dp, const Launch &L, cudaStream_t st) {
  sort_kernel<<<L.sms, kSortThreads, 0, st>>>(dp);
  gather_kernel<<<L.sms * 4, 256, 0, st>>>(dp);
}

}  // namespace tabi
