// Overlap and gutter counter of packed atlases: the paper's quality check
// (App. B: texels covered by two or more charts, with and without a 1-px
// gutter dilation) on the device, for any packing and behind every served
// batch.
//
// A texel (c, r) is covered by a placed chart iff its open square
// (c, c+1) x (r, r+1) meets the closed polygon: some edge meets the open
// square, or the square's centre lies inside (crossing parity, half-open
// in y).  The chart is drawn by its placement record (translate, rotate,
// reflect, scale by the record's own k, mirror) in units of 2^-18 texel.
// Its dilated cover is the cover grown by g texels (Chebyshev) and placed
// in the padded atlas (W + 2g) x (H + 2g), as the packer's gutters are.
//
// Row by row, exactly: in texel row J (the open band c < y < d), an edge
// that meets the band covers the columns whose open x-interval meets the
// x-range of the edge's part inside the band -- an interval whose ends
// are the edge's x at the band's bounding lines (or at its endpoints),
// floor and ceiling of exact rationals -- and a point (a vertical edge)
// covers the column whose open interval holds it.  The centres inside are
// those with an odd number of the row's centre-line crossings to their
// left; only the floor of each crossing decides that for an integer
// centre, so every crossing toggles one bit (the first column whose
// centre lies right of it) and a prefix exclusive-or along the row turns
// the toggles into the inside columns.  The row's cover is the union.
//
// Marking: per atlas four bit planes -- plain covers (W x H) occupied and
// hit twice, dilated covers (padded grid) occupied and hit twice.  A warp
// takes a block of a chart's dilated rows; its rows are kept as bit masks
// aligned to the atlas's 32-bit words in shared memory, a ring of the last
// 2g + 1 cover rows giving the dilation (the rows' union, each spread g
// bits either way).  Each word of a row goes to the plane with one
// atomicOr; bits that were already set go to the "twice" plane.  A chart's
// rows are disjoint across its warps and a word is written once per row,
// so only two charts can set a bit twice.  The counts are the bits each
// "twice" plane gains (counted as they are first set) and the cover texels
// that fall outside the atlas.
#include <mutex>

#include "context.h"

namespace tabi {

namespace {

constexpr int kCheckWarps = 8;
constexpr int kCheckThreads = 32 * kCheckWarps;
constexpr int kRowBlock = 32;  // dilated rows per work item
// words of one row mask: the widest chart (8192 columns), the alignment to
// the atlas's words (up to 31 + g bits before column 0) and the dilated
// cover's 2g columns after it
constexpr int kRowWords = (kMaxAtlas + 3 * kMaxGutter + 31) / 32 + 2;

__device__ __forceinline__ int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }

// floor(a / b), b != 0
__device__ __forceinline__ int64_t floordiv(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

// The chart's vertex i in 2^-18 texel units relative to its box (see the
// file comment), from the transform constants.
struct PlacedXf {
  int32_t minx, miny, W0, Wq, Hq, k, w;
  int rot, fx, fy, mir;
  __device__ __forceinline__ void at(const int32_t *v, int i, int64_t &X, int64_t &Y) const {
    int64_t px = v[2 * i] - minx, py = v[2 * i + 1] - miny;
    if (rot) { const int64_t t = px; px = py; py = W0 - t; }
    if (fy) py = Hq - py;
    if (fx) px = Wq - px;
    X = px * k;
    Y = py * k;
    if (mir) X = (int64_t)w * kFix - X;
  }
};

__device__ __forceinline__ unsigned long long warp_sum_ull(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Columns i0..i1 (clamped to the chart's 0..w-1) of a row mask whose bit
// px + i is column i.
__device__ __forceinline__ void or_cols(uint32_t *row, int32_t px, int64_t i0, int64_t i1, int32_t w) {
  i0 = imax(i0, 0);
  i1 = imin(i1, (int64_t)w - 1);
  if (i0 > i1) return;
  const int32_t p0 = px + (int32_t)i0, p1 = px + (int32_t)i1;
  const int t0 = p0 >> 5, t1 = p1 >> 5;
  for (int t = t0; t <= t1; ++t) {
    uint32_t m = ~0u;
    if (t == t0) m &= ~0u << (p0 & 31);
    if (t == t1) m &= ~0u >> (31 - (p1 & 31));
    atomicOr(row + t, m);
  }
}

// x(y) of the edge as n + f with n = floor, f in [0, 1); returns n and
// whether f > 0.
__device__ __forceinline__ int64_t x_at(int64_t x0, int64_t y0, int64_t dx, int64_t dy, int64_t y, bool &frac) {
  const int64_t num = (y - y0) * dx;
  const int64_t q = floordiv(num, dy);
  frac = q * dy != num;
  return x0 + q;
}

// The start of a cover row: `row` and the toggles `tog` cleared.
__device__ __forceinline__ void row_begin(uint32_t *row, uint32_t *tog, int nwr, int lane) {
  for (int t = lane; t < nwr; t += 32) {
    row[t] = 0;
    tog[t] = 0;
  }
  __syncwarp();
}

// The edge's covered columns in the band and its centre-line crossing.
// Given the edge with y0 <= y1 (endpoints in either order: the segment and
// the crossing rule are symmetric), x at the band's top line (nc + fc),
// at its centre line (floor ny) and at its bottom line (nd + fd), where
// those lines cross the edge's y-range.
__device__ __noinline__ void edge_in_band(int64_t x0, int64_t y0, int64_t x1, int64_t y1, int64_t c,
                                             int64_t nc, bool fc, int64_t ny, int64_t nd, bool fd, int32_t w,
                                             int32_t px, uint32_t *row, uint32_t *tog) {
  const int64_t d = c + kFix, cy = c + kFix / 2;
  if (y1 <= c || y0 >= d) return;  // misses the band (and its centre line)
  const int64_t dx = x1 - x0;
  if (y0 == y1) {
    if (dx != 0) {  // inside the open band: the closed x-range [lo, hi]
      const int64_t lo = imin(x0, x1), hi = imax(x0, x1);
      or_cols(row, px, lo >> 18, ((hi + kFix - 1) >> 18) - 1, w);
    }
    return;
  }
  if (dx == 0) {  // a point of x = x0: the column holding it, unless on a grid line
    if (x0 & (kFix - 1)) or_cols(row, px, x0 >> 18, x0 >> 18, w);
  } else {
    // the part inside the band runs from y = max(y0, c) to min(y1, d)
    const int64_t nA = y0 > c ? x0 : nc, nB = y1 < d ? x1 : nd;
    const bool fA = y0 > c ? false : fc, fB = y1 < d ? false : fd;
    const bool up = dx > 0;  // x grows with y
    const int64_t nlo = up ? nA : nB, nhi = up ? nB : nA;
    const bool fhi = up ? fB : fA;
    // columns whose open interval meets (inf, sup): floor(inf) .. ceil(sup) - 1
    or_cols(row, px, nlo >> 18, (fhi ? (nhi >> 18) + 1 : (nhi + kFix - 1) >> 18) - 1, w);
  }
  if (y0 <= cy && cy < y1) {  // crosses the centre line: toggle at the first centre right of it
    int64_t t = ((ny >> 17) + 1) >> 1;
    t = imin(imax(t, 0), w);
    const int32_t p = px + (int32_t)t;
    atomicXor(tog + (p >> 5), 1u << (p & 31));
  }
}

// The end of a cover row: the prefix exclusive-or of the toggles (the
// inside columns) joined to the edges' columns.
__device__ __forceinline__ void row_finish(uint32_t *row, const uint32_t *tog, int nwr, int lane) {
  __syncwarp();
  uint32_t carry = 0;
  for (int t0 = 0; t0 < nwr; t0 += 32) {
    const int t = t0 + lane;
    uint32_t x = t < nwr ? tog[t] : 0u;
    x ^= x << 1;
    x ^= x << 2;
    x ^= x << 4;
    x ^= x << 8;
    x ^= x << 16;
    const unsigned par = __ballot_sync(0xffffffffu, (x >> 31) & 1u);
    if (((__popc(par & ((1u << lane) - 1u)) & 1u) ^ carry) != 0u) x = ~x;
    if (t < nwr && x) row[t] |= x;
    carry ^= __popc(par) & 1u;
  }
  __syncwarp();
}

// Cover row J of the chart (0 <= J < h) into `row` (nwr words, bit px + i
// = column i), any number of vertices: each edge's x at the band's lines
// by exact division.
__device__ __noinline__ void cover_row(const PlacedXf &xf, const int32_t *v, int nv, int32_t J, int32_t w,
                                       int32_t px, int nwr, uint32_t *row, uint32_t *tog, int lane) {
  auto vert = [&xf, v](int e, int64_t &x, int64_t &y) { xf.at(v, e, x, y); };
  row_begin(row, tog, nwr, lane);
  const int64_t c = (int64_t)J * kFix;
  for (int e = lane; e < nv; e += 32) {
    int64_t x0, y0, x1, y1;
    vert(e == 0 ? nv - 1 : e - 1, x0, y0);
    vert(e, x1, y1);
    if (y0 > y1) {
      int64_t t = x0; x0 = x1; x1 = t;
      t = y0; y0 = y1; y1 = t;
    }
    if (y1 <= c || y0 >= c + kFix) continue;
    int64_t nc = 0, ny = 0, nd = 0;
    bool fc = false, fd = false, fy;
    if (y1 > y0) {
      nc = x_at(x0, y0, x1 - x0, y1 - y0, c, fc);
      ny = x_at(x0, y0, x1 - x0, y1 - y0, c + kFix / 2, fy);
      nd = x_at(x0, y0, x1 - x0, y1 - y0, c + kFix, fd);
    }
    edge_in_band(x0, y0, x1, y1, c, nc, fc, ny, nd, fd, w, px, row, tog);
  }
  row_finish(row, tog, nwr, lane);
}

// An edge of a chart with at most 64 vertices kept by its lane across the
// rows: endpoints with y0 <= y1 and x at the half-row lines y = m F / 2 as
// x0 + q + r / dy (0 <= r < dy), stepped exactly from line to line by the
// quotient and remainder of F / 2 * dx / dy -- no division per row.
struct EdgeDDA {
  int64_t x0, y0, x1, y1, dy, qh, rh, q, r;
  __device__ __forceinline__ void init(int64_t ax, int64_t ay, int64_t bx, int64_t by, int32_t J) {
    if (ay > by) {
      x0 = bx; y0 = by; x1 = ax; y1 = ay;
    } else {
      x0 = ax; y0 = ay; x1 = bx; y1 = by;
    }
    dy = y1 - y0;
    if (dy > 0) {
      const int64_t dx = x1 - x0;
      qh = floordiv((kFix / 2) * dx, dy);
      rh = (kFix / 2) * dx - qh * dy;
      const int64_t num = ((int64_t)J * kFix - y0) * dx;
      q = floordiv(num, dy);
      r = num - q * dy;
    }
  }
  __device__ __forceinline__ void step() {
    q += qh;
    r += rh;
    if (r >= dy) {
      r -= dy;
      ++q;
    }
  }
};

// Cover row J from the lanes' edges (at most two each); the edges' state
// is at row J on entry and at row J + 1 on return.
__device__ __forceinline__ void cover_row_dda(EdgeDDA (&ed)[2], int ne, int32_t J, int32_t w, int32_t px,
                                              int nwr, uint32_t *row, uint32_t *tog, int lane) {
  row_begin(row, tog, nwr, lane);
  const int64_t c = (int64_t)J * kFix;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    if (s >= ne) break;
    EdgeDDA &E = ed[s];
    const bool meets = E.y1 > c && E.y0 < c + kFix;  // the edge meets the band
    if (E.dy > 0) {
      const int64_t nc = E.x0 + E.q;
      const bool fc = E.r != 0;
      E.step();
      const int64_t ny = E.x0 + E.q;
      E.step();
      if (meets) edge_in_band(E.x0, E.y0, E.x1, E.y1, c, nc, fc, ny, E.x0 + E.q, E.r != 0, w, px, row, tog);
    } else if (meets) {
      edge_in_band(E.x0, E.y0, E.x1, E.y1, c, 0, false, 0, 0, false, w, px, row, tog);
    }
  }
  row_finish(row, tog, nwr, lane);
}

// Bits of the 32-column word starting at atlas column X0 that lie in [0, lim).
__device__ __forceinline__ uint32_t valid_bits(int64_t X0, int64_t lim) {
  if (X0 >= 0 && X0 + 32 <= lim) return ~0u;
  const int64_t lo = imax(0, -X0), hi = imin(32, lim - X0);
  if (lo >= hi) return 0u;
  const uint32_t up = hi >= 32 ? ~0u : ((1u << hi) - 1u);
  return up & (~0u << lo);
}

__global__ void check_clear_kernel(uint32_t *p, int64_t words) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0;
}

// A chart's placed box, from its vertices (check_size_kernel).
struct CheckChart {
  int32_t minx, miny, W0, Wq, Hq, w, h, a;  // a: its atlas
};

// Per chart (a warp each): its box at its placement's scale and its number
// of blocks of kRowBlock dilated rows (0: not drawn -- its atlas has no
// planes, fewer than three vertices, a scale outside 1..1024), counted in
// nblk[0 .. N) for charts of at most 64 vertices and in nblk[N + 1 ..
// 2N + 1) for larger ones (each mark kernel walks its own units).
__global__ void __launch_bounds__(kCheckThreads) check_size_kernel(const CheckAtlas *__restrict__ atl,
                                                                   const int32_t *__restrict__ catl, int64_t N,
                                                                   int gmax, CheckChart *__restrict__ cc,
                                                                   int64_t *__restrict__ nblk) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t gc = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; gc < N; gc += nw) {
    const int a = catl ? catl[gc] : 0;
    const CheckAtlas &ca = atl[a];
    const int c = (int)(gc - ca.cb);
    const uint32_t o0 = ca.offsets[c], o1 = ca.offsets[c + 1];
    const tabi_placement pl = ca.place[c];
    if (ca.plane0 < 0 || ca.g > gmax || o1 < o0 + 3 || pl.k < 1 || pl.k > 1024) {
      if (lane == 0) nblk[gc] = nblk[N + 1 + gc] = 0;
      continue;
    }
    const int nv = (int)(o1 - o0);
    const int32_t *v = ca.verts + 2 * (int64_t)o0;
    int32_t mnx = 0x7fffffff, mny = 0x7fffffff, mxx = -0x7fffffff - 1, mxy = -0x7fffffff - 1;
    for (int i = lane; i < nv; i += 32) {
      mnx = min(mnx, v[2 * i]); mxx = max(mxx, v[2 * i]);
      mny = min(mny, v[2 * i + 1]); mxy = max(mxy, v[2 * i + 1]);
    }
    mnx = warp_min(mnx); mxx = warp_max(mxx); mny = warp_min(mny); mxy = warp_max(mxy);
    if (lane == 0) {
      CheckChart r;
      r.minx = mnx;
      r.miny = mny;
      r.W0 = mxx - mnx;
      r.Wq = pl.rot90 ? mxy - mny : r.W0;
      r.Hq = pl.rot90 ? r.W0 : mxy - mny;
      r.w = (int32_t)(((int64_t)r.Wq * pl.k + kFix - 1) >> 18);
      r.h = (int32_t)(((int64_t)r.Hq * pl.k + kFix - 1) >> 18);
      r.a = a;
      cc[gc] = r;
      const int64_t b = r.w > kMaxAtlas ? 0 : (r.h + 2 * ca.g + kRowBlock - 1) / kRowBlock;
      const bool small = o1 - o0 <= 64;
      nblk[gc] = small ? b : 0;
      nblk[N + 1 + gc] = small ? 0 : b;
    }
  }
}

// Exclusive prefix sum of v[0..N) in place, v[N] = the total (one block of
// 1024 threads, each a contiguous run); block b scans the array at v + b (N + 1).
__global__ void __launch_bounds__(1024) check_scan_kernel(int64_t *v, int64_t N) {
  v += blockIdx.x * (N + 1);
  __shared__ int64_t wsum[32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int64_t run = (N + 1023) / 1024, b = (int64_t)t * run, e = b + run < N ? b + run : N;
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += v[i];
  int64_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int64_t x = wsum[lane], xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += y;
    }
    wsum[lane] = xi - x;  // exclusive over the warps
  }
  __syncthreads();
  int64_t base = wsum[wid] + incl - s;
  for (int64_t i = b; i < e; ++i) {
    const int64_t x = v[i];
    v[i] = base;
    base += x;
  }
  if (t == 1023) v[N] = base;
}

// The chart holding unit u: the largest c with off[c] <= u (off[0] = 0 <=
// u < off[N]), the warp probing 32 positions a step.
__device__ __forceinline__ int64_t unit_chart(const int64_t *__restrict__ off, int64_t N, int64_t u, int lane) {
  int64_t lo = 0, hi = N;  // off[lo] <= u < off[hi]
  while (hi - lo > 32) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t pos = lo + lane * step;
    const unsigned m = __ballot_sync(0xffffffffu, pos < hi && off[pos] <= u);
    lo += (31 - __clz(m)) * step;
    hi = lo + step < hi ? lo + step : hi;
  }
  const int64_t pos = lo + lane;
  const unsigned m = __ballot_sync(0xffffffffu, pos < hi && off[pos] <= u);
  return lo + 31 - __clz(m);
}

// Units: (chart, block of kRowBlock dilated rows), balanced over the warps.
// Shared memory per warp: the ring of 2g + 1 cover rows and one scratch
// row, kRowWords words each.
// kDDA: the units of charts of at most 64 vertices (edges stepped down the
// rows, two blocks per multiprocessor), else those of larger charts.
template <bool kDDA>
__global__ void __launch_bounds__(kCheckThreads, kDDA ? 2 : 1)
    check_mark_kernel(const CheckAtlas *__restrict__ atl, const CheckChart *__restrict__ cc,
                      const int64_t *__restrict__ off, int64_t N, int gmax, uint32_t *planes,
                      unsigned long long *counts) {
  extern __shared__ uint32_t csm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint32_t *ring = csm + (size_t)wib * (2 * gmax + 2) * kRowWords;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = off[N];
  for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < total; u += nw) {
    const int64_t gc = unit_chart(off, N, u, lane);
    const int blk = (int)(u - off[gc]);
    const CheckChart r = cc[gc];
    const int a = r.a;
    const CheckAtlas &ca = atl[a];
    const int c = (int)(gc - ca.cb);
    const uint32_t o0 = ca.offsets[c];
    const int nv = (int)(ca.offsets[c + 1] - o0);
    const int32_t *v = ca.verts + 2 * (int64_t)o0;
    const tabi_placement pl = ca.place[c];
    PlacedXf xf;
    xf.minx = r.minx; xf.miny = r.miny; xf.W0 = r.W0; xf.Wq = r.Wq; xf.Hq = r.Hq;
    xf.rot = pl.rot90; xf.fx = pl.flip_x; xf.fy = pl.flip_y; xf.mir = pl.mirror;
    xf.k = pl.k;
    xf.w = r.w;
    const int32_t w = r.w, h = r.h;
    const int g = ca.g, S = 2 * g + 1;
    // row masks aligned to the atlas's words: bit px + i is column i
    const int64_t base = ((int64_t)pl.x - g) & ~(int64_t)31;
    const int32_t px = (int32_t)(pl.x - base);
    const int nwr = ((px + w + 2 * g) >> 5) + 1;  // up to the dilated cover's last bit
    uint32_t *tog = ring + (size_t)S * kRowWords;
    auto vert = [&xf, v](int e, int64_t &x, int64_t &y) { xf.at(v, e, x, y); };
    // up to 64 vertices: each lane keeps its (at most two) edges and steps
    // them down the rows from the block's first cover row
    const int32_t J0 = -g + blk * kRowBlock, J1 = min(J0 + kRowBlock, h + g);
    EdgeDDA ed[2];
    int ne = 0;
    if (kDDA) {
      const int32_t Jstart = max(J0 - g, 0);
#pragma unroll
      for (int s2 = 0; s2 < 2; ++s2) {
        const int e = lane + 32 * s2;
        if (e < nv) {
          int64_t ax, ay, bx, by;
          vert(e == 0 ? nv - 1 : e - 1, ax, ay);
          vert(e, bx, by);
          ed[s2].init(ax, ay, bx, by, Jstart);
          ne = s2 + 1;
        }
      }
    }
    int ld = 0;  // the ring slot the next cover row goes to
    auto load_row = [&](int32_t J) {  // cover row J (zero outside the chart)
      uint32_t *rw = ring + (size_t)ld * kRowWords;
      ld = ld + 1 == S ? 0 : ld + 1;
      if (J >= 0 && J < h) {
        if (kDDA)
          cover_row_dda(ed, ne, J, w, px, nwr, rw, tog, lane);
        else
          cover_row(xf, v, nv, J, w, px, nwr, rw, tog, lane);
      } else {
        for (int t = lane; t < nwr; t += 32) rw[t] = 0;
        __syncwarp();
      }
    };
    uint32_t *pocc = planes + ca.plane0, *ptwice = pocc + (int64_t)ca.wpp * ca.H;
    uint32_t *docc = ptwice + (int64_t)ca.wpp * ca.H, *dtwice = docc + (int64_t)ca.wpd * (ca.H + 2 * g);
    unsigned long long outside = 0, twice_p = 0, twice_d = 0;
    for (int32_t J = J0 - g; J < J0 + g; ++J) load_row(J);
    int mid = g;  // the ring slot of the dilated row's own cover row
    for (int32_t Jd = J0; Jd < J1; ++Jd) {
      load_row(Jd + g);
      const int64_t Y = (int64_t)pl.y + Jd;
      const uint32_t *cen = ring + (size_t)mid * kRowWords;
      for (int t = lane; t < nwr; t += 32) {
        const int64_t X0 = base + 32 * (int64_t)t;
        // the plain cover, texels (x + i, y + Jd)
        uint32_t pm = 0;
        if (Jd >= 0 && Jd < h) {
          const uint32_t m = cen[t];
          const uint32_t ok = (Y >= 0 && Y < ca.H) ? valid_bits(X0, ca.W) : 0u;
          outside += __popc(m & ~ok);
          pm = m & ok;
        }
        // the dilated cover in the padded atlas: chart column i, row Jd
        // (-g <= i < w + g) is padded texel (x + i + g, y + Jd + g), the
        // union of the cover rows Jd - g .. Jd + g (the whole ring), each
        // spread g columns either way -- here shifted by 0 .. 2g bits up
        // (the spread of a union is the union of the spreads: the rows are
        // joined first and spread once)
        uint32_t cur = 0, prv = 0;
        for (int sl = 0; sl < S; ++sl) {
          const uint32_t *rw = ring + (size_t)sl * kRowWords;
          cur |= rw[t];
          prv |= t > 0 ? rw[t - 1] : 0u;
        }
        uint32_t dm = cur;
        for (int q = 1; q <= 2 * g; ++q) dm |= (cur << q) | (prv >> (32 - q));
        const int64_t Yd = Y + g;
        dm = (Yd >= 0 && Yd < ca.H + 2 * g) ? dm & valid_bits(X0, ca.W + 2 * g) : 0u;
        // both words' atomics in flight together; the bits already set go
        // to the "twice" planes
        const int64_t ip = Y * ca.wpp + (X0 >> 5), id = Yd * ca.wpd + (X0 >> 5);
        const uint32_t op = pm ? atomicOr(pocc + ip, pm) : 0u;
        const uint32_t od = dm ? atomicOr(docc + id, dm) : 0u;
        // a bit newly set in a "twice" plane is a texel counted once
        if (op & pm) twice_p += __popc(op & pm & ~atomicOr(ptwice + ip, op & pm));
        if (od & dm) twice_d += __popc(od & dm & ~atomicOr(dtwice + id, od & dm));
      }
      mid = mid + 1 == S ? 0 : mid + 1;
      __syncwarp();
    }
    outside = warp_sum_ull(outside);
    twice_p = warp_sum_ull(twice_p);
    twice_d = warp_sum_ull(twice_d);
    if (lane == 0) {
      if (twice_p) atomicAdd(counts + 3 * a + 0, twice_p);
      if (twice_d) atomicAdd(counts + 3 * a + 1, twice_d);
      if (outside) atomicAdd(counts + 3 * a + 2, outside);
    }
  }
}

// The counts of an atlas without planes: all ~0 (unchecked).  The others
// were counted by the mark kernels as their "twice" bits were first set.
__global__ void check_count_kernel(const CheckAtlas *__restrict__ atl, int A, unsigned long long *counts) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < A; a += gridDim.x * blockDim.x)
    if (atl[a].plane0 < 0) counts[3 * a + 0] = counts[3 * a + 1] = counts[3 * a + 2] = ~0ull;
}

}  // namespace

int64_t check_plane_words(int W, int H, int g) {
  const int64_t wpp = (W + 31) / 32, wpd = (W + 2 * g + 31) / 32;
  return 2 * wpp * H + 2 * wpd * (H + 2 * g);
}

void fill_check_atlas(CheckAtlas &ca, int W, int H, int g) {
  ca.W = W;
  ca.H = H;
  ca.g = g;
  ca.wpp = (W + 31) / 32;
  ca.wpd = (W + 2 * g + 31) / 32;
}

size_t check_scratch_bytes(int64_t N) {
  return ((sizeof(CheckChart) * (size_t)N + 255) & ~(size_t)255) + ((16 * ((size_t)N + 1) + 255) & ~(size_t)255);
}

// Clears the planes, sizes every chart, lays the (chart, row block) units
// out, marks them, counts; `counts` (3 per atlas: plain texels hit twice,
// dilated texels hit twice, cover texels outside the atlas) must be zero
// on entry.
void launch_check(const CheckAtlas *datl, int A, const int32_t *catl, int64_t N, int gmax, uint32_t *planes,
                  int64_t words, void *scratch, unsigned long long *counts, int sms, cudaStream_t st) {
  static std::once_flag attr;
  std::call_once(attr, [] {  // the most the gutter limit needs
    const int most = (int)(sizeof(uint32_t) * kCheckWarps * (2 * kMaxGutter + 2) * kRowWords);
    cudaFuncSetAttribute(check_mark_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    cudaFuncSetAttribute(check_mark_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  });
  CheckChart *cc = reinterpret_cast<CheckChart *>(scratch);
  int64_t *off = reinterpret_cast<int64_t *>(reinterpret_cast<char *>(scratch) +
                                             ((sizeof(CheckChart) * (size_t)N + 255) & ~(size_t)255));
  const size_t smem = sizeof(uint32_t) * kCheckWarps * (2 * (size_t)gmax + 2) * kRowWords;
  check_clear_kernel<<<sms * 4, 256, 0, st>>>(planes, words);
  check_size_kernel<<<sms * 4, kCheckThreads, 0, st>>>(datl, catl, N, gmax, cc, off);
  check_scan_kernel<<<2, 1024, 0, st>>>(off, N);
  check_mark_kernel<true><<<sms * 2, kCheckThreads, smem, st>>>(datl, cc, off, N, gmax, planes, counts);
  check_mark_kernel<false><<<sms, kCheckThreads, smem, st>>>(datl, cc, off + N + 1, N, gmax, planes, counts);
  check_count_kernel<<<(A + 255) / 256, 256, 0, st>>>(datl, A, counts);
}

}  // namespace tabi
