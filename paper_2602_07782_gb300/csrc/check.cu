// Overlap and gutter counter of packed atlases: the paper's quality check
// (App. B: texels covered by two or more charts, with and without a 1-px
// gutter dilation) on the device, for any packing and behind every served
// batch.
//
// A texel (c, r) is covered by a placed chart iff its open square
// (c, c+1) x (r, r+1) meets the closed polygon: some edge meets the open
// square (separating axes x, y and the edge normal, in exact integers) or
// the square's centre lies inside (crossing parity, half-open in y).  The
// chart is drawn by its placement record (translate, rotate, reflect,
// scale by the record's own k, mirror) in units of 2^-18 texel.  Its
// dilated cover is the cover grown by g texels (Chebyshev) and placed in
// the padded atlas (W + 2g) x (H + 2g), as the packer's gutters are.
//
// Marking: per atlas four bit planes -- plain covers (W x H) occupied and
// hit twice, dilated covers (padded grid) occupied and hit twice.  A warp
// draws one chart, lane l taking texel column base - 2g + l of the cover;
// rows run down the chart, a (2g+1)-row shift register per lane and
// shuffles from the 2g lanes to the left give the dilation, and the lanes
// that meet one bit-plane word join their bits (__match_any_sync) into one
// atomicOr; bits that were already set go to the "twice" plane.  A chart's
// own texels are distinct, so only two charts can set a bit twice.  The
// counts are the population counts of the "twice" planes and the cover
// texels that fall outside the atlas.
#include "context.h"

namespace tabi {

namespace {

constexpr int kCheckThreads = 256;

__device__ __forceinline__ int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }


constexpr int kWarpVerts = 128;   // vertices a warp keeps transformed in shared memory
constexpr int kChunkSplit = 8;    // warps sharing one chart's column chunks

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

// Is texel (i, j) of the chart's box covered?  vert(e, x, y) gives the
// transformed vertex e (nv of them).  Coordinates are below 2^31 in size (chart extents below
// 2^21 in 1/256 texel, k <= 1024), so every product of two differences
// stays below 2^62.  Edges whose y-range misses the texel row's band and
// its centre line are skipped (the row is the same for the whole warp).
template <class Get>
__device__ bool covered(const Get &vert, int nv, int32_t i, int32_t j) {
  const int64_t a = (int64_t)i * kFix, b = a + kFix, c = (int64_t)j * kFix, d = c + kFix;
  const int64_t cx = (2 * (int64_t)i + 1) * (kFix / 2), cy = (2 * (int64_t)j + 1) * (kFix / 2);
  bool inside = false;
  int64_t x0, y0;
  vert(nv - 1, x0, y0);
  for (int e = 0; e < nv; ++e) {
    int64_t x1, y1;
    vert(e, x1, y1);
    const int64_t ylo = imin(y0, y1), yhi = imax(y0, y1);
    if (yhi > c && ylo < d && (x0 != x1 || y0 != y1)) {
      const int64_t dx = x1 - x0, dy = y1 - y0;
      if (!(imax(x0, x1) <= a || imin(x0, x1) >= b)) {
        const int64_t s1 = dx * (c - y0) - dy * (a - x0), s2 = dx * (c - y0) - dy * (b - x0);
        const int64_t s3 = dx * (d - y0) - dy * (a - x0), s4 = dx * (d - y0) - dy * (b - x0);
        const bool allpos = s1 >= 0 && s2 >= 0 && s3 >= 0 && s4 >= 0;
        const bool allneg = s1 <= 0 && s2 <= 0 && s3 <= 0 && s4 <= 0;
        if (!allpos && !allneg) return true;  // the edge meets the open square
      }
    }
    if ((y0 > cy) != (y1 > cy)) {  // crosses the centre's line (half-open in y)
      const int64_t dx = x1 - x0, dy = y1 - y0;
      const int64_t l = (cx - x0) * dy, r = (cy - y0) * dx;
      const bool right_of = dy > 0 ? l > r : l < r;
      inside ^= !right_of;
    }
    x0 = x1;
    y0 = y1;
  }
  return inside;
}

// Set the lanes' bits (one texel each, `on`) in a plane of `wpr` words per
// row: lanes meeting one word join their bits; bits already set go to
// `twice`.
__device__ __forceinline__ void mark(uint32_t *occ, uint32_t *twice, bool on, int64_t X, int64_t Y, int wpr) {
  const int64_t word = on ? Y * wpr + (X >> 5) : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, word);
  const uint32_t m = __reduce_or_sync(peers, on ? 1u << (X & 31) : 0u);
  if (on && (int)(threadIdx.x & 31) == __ffs(peers) - 1) {
    const uint32_t old = atomicOr(occ + word, m);
    if (old & m) atomicOr(twice + word, old & m);
  }
}

__global__ void check_clear_kernel(uint32_t *p, int64_t words) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0;
}

// Items: (chart, split q): the warp draws the chart's column chunks q,
// q + kChunkSplit, ... (a chunk: 32 - 2g dilated columns, all rows).
__global__ void __launch_bounds__(kCheckThreads) check_mark_kernel(const CheckAtlas *__restrict__ atl, int A,
                                                                   const int32_t *__restrict__ catl, int64_t N,
                                                                   uint32_t *planes, unsigned long long *counts) {
  __shared__ int64_t sx[kCheckThreads / 32][kWarpVerts], sy[kCheckThreads / 32][kWarpVerts];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t item = gw; item < N * kChunkSplit; item += nw) {
    const int64_t gc = item / kChunkSplit;
    const int q = (int)(item % kChunkSplit);
    const int a = catl ? catl[gc] : 0;
    const CheckAtlas &ca = atl[a];
    if (ca.plane0 < 0) continue;  // no room for its planes
    const int c = (int)(gc - ca.cb);
    const uint32_t o0 = ca.offsets[c], o1 = ca.offsets[c + 1];
    if (o1 < o0 + 3) continue;
    const int nv = (int)(o1 - o0);
    const int32_t *v = ca.verts + 2 * (int64_t)o0;
    const tabi_placement pl = ca.place[c];
    if (pl.k < 1 || pl.k > 1024) continue;
    int32_t mnx = 0x7fffffff, mny = 0x7fffffff, mxx = -0x7fffffff - 1, mxy = -0x7fffffff - 1;
    for (int i = lane; i < nv; i += 32) {
      mnx = min(mnx, v[2 * i]); mxx = max(mxx, v[2 * i]);
      mny = min(mny, v[2 * i + 1]); mxy = max(mxy, v[2 * i + 1]);
    }
    mnx = warp_min(mnx); mxx = warp_max(mxx); mny = warp_min(mny); mxy = warp_max(mxy);
    PlacedXf xf;
    xf.minx = mnx; xf.miny = mny; xf.W0 = mxx - mnx;
    xf.rot = pl.rot90; xf.fx = pl.flip_x; xf.fy = pl.flip_y; xf.mir = pl.mirror;
    xf.Wq = xf.rot ? mxy - mny : xf.W0;
    xf.Hq = xf.rot ? xf.W0 : mxy - mny;
    xf.k = pl.k;
    const int32_t w = (int32_t)(((int64_t)xf.Wq * xf.k + kFix - 1) >> 18);
    const int32_t h = (int32_t)(((int64_t)xf.Hq * xf.k + kFix - 1) >> 18);
    xf.w = w;
    const int g = ca.g;
    const int step = 32 - 2 * g;
    const int nchunks = (w + 2 * g + step - 1) / step;
    if (q >= nchunks) continue;
    // the transformed vertices in shared memory if they fit; larger charts
    // transform them from the input at every texel
    const bool shared = nv <= kWarpVerts;
    __syncwarp();
    if (shared)
      for (int i = lane; i < nv; i += 32) xf.at(v, i, sx[wib][i], sy[wib][i]);
    __syncwarp();
    const int64_t *xs = sx[wib], *ys = sy[wib];
    auto from_shared = [xs, ys](int e, int64_t &x, int64_t &y) { x = xs[e]; y = ys[e]; };
    auto from_input = [&xf, v](int e, int64_t &x, int64_t &y) { xf.at(v, e, x, y); };
    uint32_t *pocc = planes + ca.plane0, *ptwice = pocc + (int64_t)ca.wpp * ca.H;
    uint32_t *docc = ptwice + (int64_t)ca.wpp * ca.H, *dtwice = docc + (int64_t)ca.wpd * (ca.H + 2 * g);
    unsigned long long outside = 0;
    for (int ch = q; ch < nchunks; ch += kChunkSplit) {
      const int32_t base = ch * step;
      const int32_t i = base - 2 * g + lane;  // this lane's cover column (dilated column for lanes >= 2g)
      const bool col = i >= 0 && i < w;
      const bool own = lane >= 2 * g && i < w + 2 * g;  // the columns this chunk outputs
      uint32_t win = 0;                                  // cover bits of the last 2g + 1 rows
      for (int32_t J = 0; J < h + 2 * g; ++J) {
        const bool cv =
            col && J < h && (shared ? covered(from_shared, nv, i, J) : covered(from_input, nv, i, J));
        win = ((win << 1) | (cv ? 1u : 0u)) & ((2u << (2 * g)) - 1u);
        bool dil = win != 0;
        for (int o = 1; o <= 2 * g; ++o) {
          const int up = __shfl_up_sync(0xffffffffu, win != 0 ? 1 : 0, o);
          dil |= lane >= o && up;
        }
        const int64_t X = (int64_t)pl.x + i, Y = (int64_t)pl.y + J;
        // the plain cover, texel (x + i, y + J)
        const bool pin = X >= 0 && X < ca.W && Y >= 0 && Y < ca.H;
        if (cv && own && !pin) ++outside;
        mark(pocc, ptwice, cv && own && pin, X, Y, ca.wpp);
        // the dilated cover, padded texel (x + i, y + J)
        const bool din = X >= 0 && X < ca.W + 2 * g && Y >= 0 && Y < ca.H + 2 * g;
        mark(docc, dtwice, dil && own && din, X, Y, ca.wpd);
      }
    }
    outside = warp_sum_ull(outside);
    if (lane == 0 && outside) atomicAdd(counts + 3 * a + 2, outside);
  }
}

// Per atlas: population counts of the two "twice" planes.
__global__ void __launch_bounds__(kCheckThreads) check_count_kernel(const CheckAtlas *__restrict__ atl, int A,
                                                                    const uint32_t *planes,
                                                                    unsigned long long *counts) {
  __shared__ unsigned long long part[2];
  for (int a = blockIdx.x; a < A; a += gridDim.x) {
    const CheckAtlas &ca = atl[a];
    if (threadIdx.x < 2) part[threadIdx.x] = 0;
    __syncthreads();
    if (ca.plane0 >= 0) {
      const int64_t np = (int64_t)ca.wpp * ca.H, nd = (int64_t)ca.wpd * (ca.H + 2 * ca.g);
      const uint32_t *ptwice = planes + ca.plane0 + np, *dtwice = ptwice + np + nd;
      unsigned long long s0 = 0, s1 = 0;
      for (int64_t i = threadIdx.x; i < np; i += blockDim.x) s0 += __popc(ptwice[i]);
      for (int64_t i = threadIdx.x; i < nd; i += blockDim.x) s1 += __popc(dtwice[i]);
      s0 = warp_sum_ull(s0);
      s1 = warp_sum_ull(s1);
      if ((threadIdx.x & 31) == 0) { atomicAdd(&part[0], s0); atomicAdd(&part[1], s1); }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      counts[3 * a + 0] = ca.plane0 >= 0 ? part[0] : ~0ull;
      counts[3 * a + 1] = ca.plane0 >= 0 ? part[1] : ~0ull;
      if (ca.plane0 < 0) counts[3 * a + 2] = ~0ull;
    }
    __syncthreads();
  }
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

// Clears the planes, marks every chart, counts; `counts` (3 per atlas:
// plain texels hit twice, dilated texels hit twice, cover texels outside
// the atlas) must be zero on entry.
void launch_check(const CheckAtlas *datl, int A, const int32_t *catl, int64_t N, uint32_t *planes, int64_t words,
                  unsigned long long *counts, int sms, cudaStream_t st) {
  check_clear_kernel<<<sms * 4, 256, 0, st>>>(planes, words);
  check_mark_kernel<<<sms * 8, kCheckThreads, 0, st>>>(datl, A, catl, N, planes, counts);
  check_count_kernel<<<sms * 2, kCheckThreads, 0, st>>>(datl, A, planes, counts);
}

}  // namespace tabi
