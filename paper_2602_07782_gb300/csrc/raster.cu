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
// Columns and rows go to per-(atlas, candidate) regions of the column and
// row pools with the charts back to back (the row loop copies a row's
// columns in one contiguous range).  A batch runs in waves of candidates;
// the regions of one wave tile the pools and the next wave reuses them.
// Every kernel here is persistent: a fixed grid loops over the work the
// wave plan left on the device (the charts of atlases still searching).
#include "raster_dev.cuh"

namespace tabi {
namespace {

constexpr int kRasterThreads = 256;
constexpr int kRasterWarps = kRasterThreads / 32;

// Warp-items: (chart of an atlas still searching, run of G consecutive
// candidates of the atlas's wave range).  G is chosen so that the wave has
// about raster_items warp-items (a tuned launch shape).
__global__ void __launch_bounds__(kRasterThreads, 3) raster_kernel(const Pack *__restrict__ pp, int q, int nj) {
  __shared__ rmath::AxisK axk[kRasterWarps][2];
  const Pack &p = *pp;
  const int wave = *(volatile const int32_t *)p.cur_wave;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t total = p.act_info[1];
  const int64_t target = p.raster_items;
  int G = (int)(((int64_t)nj * total + target - 1) / target);
  G = G < 1 ? 1 : (G > nj ? nj : G);
  const int ngroups = (nj + G - 1) / G;
  const uint32_t items = (uint32_t)(total * ngroups);  // about raster_items, or one per chart: below 2^31
  const int64_t N = p.N;
  const bool use_l = (p.flags & TABI_F_LAABB) != 0, use_o = (p.flags & TABI_F_OBB) != 0;
  const bool all = q == 0 || (p.flags & TABI_F_EVAL_ALL);  // later chunks: running candidates only
  const int g = p.g;
  rmath::AxisK &a0 = axk[wib][0], &a1 = axk[wib][1];
  __shared__ unsigned long long cta_words[2];  // scanline and column words of this CTA (one global add)
  if (threadIdx.x < 2) cta_words[threadIdx.x] = 0;
  __syncthreads();
  // items go to warps as they free up (a device counter per (wave, chunk)):
  // an item's cost follows its chart's size, which spans orders of
  // magnitude, so a fixed assignment leaves most warps idle behind the few
  // that drew the largest charts
  uint32_t *next_item = p.rcounter + wave * kChunkSlots + q;
  while (true) {
    uint32_t grab = 0;
    if (lane == 0) grab = atomicAdd(next_item, 1u);
    const uint32_t it = __shfl_sync(0xffffffffu, grab, 0);
    if (it >= items) break;
    const int4 e = p.act_ext[it / (uint32_t)ngroups];  // chart, atlas, top candidate, first chart
    const int s = e.x, at = e.y;
    const int cb = e.w & 0x7fffffff;
    const WaveRange wr = wave_range(e.z, wave, nj);
    const int j0 = wr.lo + (int)(it % (uint32_t)ngroups) * G;
    const int j1 = min(j0 + G, wr.hi + 1);
    if (j0 >= j1) continue;  // this atlas has fewer candidates left than the wave
    const ChartShape &sh = p.shape[s];
    const int m = sh.m;
    const int64_t C = kObbCos[m], S = kObbSin[m];
    // lanes 24-31 carry the eight corner quantities across the candidates
    rmath::CornerQ cq;
    const bool corner_lane = lane >= 24 && use_o && m > 0;
    // per chart, kept across the run of candidates: the piece lanes' slice
    // bounds and their cross slice's extent and bounds (registers) and the
    // OBB lanes' scale-free terms (shared).  Lane i < 10 holds x-slice slot
    // i as a column piece and y-slice slot i as a column cross piece; lane
    // 10 + i the same with the axes swapped.  A cross slot's bounds are
    // those of its K-slice: slot i holds slice s = i K / 10, whose bounds
    // are the ten-slot boundaries 10 s / K and 10 (s + 1) / K.
    uint32_t pb0 = 0, pb1 = 0, plq = 0, phq = 0, ce0 = 0, ce1 = 0, cb0 = 0, cb1 = 0;
    if (lane < 2 * rmath::kK) {
      const int ax = lane >= rmath::kK, i = lane - ax * rmath::kK;
      const uint32_t ext = (uint32_t)(ax ? sh.Hq : sh.Wq), oth = (uint32_t)(ax ? sh.Wq : sh.Hq);
      pb0 = i * ext / rmath::kK;
      pb1 = (i + 1) * ext / rmath::kK;
      plq = (uint32_t)(ax ? sh.xlo[i] : sh.ylo[i]);
      phq = (uint32_t)(ax ? sh.xhi[i] : sh.yhi[i]);
      ce0 = (uint32_t)(ax ? sh.ylo[i] : sh.xlo[i]);
      ce1 = (uint32_t)(ax ? sh.yhi[i] : sh.xhi[i]);
      const int sl = i * p.laabb_k / rmath::kK;
      cb0 = (uint32_t)(sl * rmath::kK / p.laabb_k) * oth / rmath::kK;
      cb1 = (uint32_t)((sl + 1) * rmath::kK / p.laabb_k) * oth / rmath::kK;
    } else if (lane < 2 * rmath::kK + 2) {
      const int ax = lane - 2 * rmath::kK;
      rmath::setup_obb_fixed(ax ? a1 : a0, ax, m, C, S, kObbDivCos[m], kObbDivSin[m], use_l, use_o);
    }
    if (corner_lane) {
      int64_t qs, rs;
      rmath::corner_step(lane - 24, C, S, sh.u0, sh.u1, sh.v0, sh.v1, qs, rs);
      rmath::corner_init(cq, lane - 24, j0, C, S, qs, rs);
    }
    for (int j = j0; j < j1; ++j) {
      const int64_t k = 16 * (j + 1);
      // a finished candidate (later chunks): nothing to draw; the corner
      // quantities still step to the next candidate
      if (!all && (p.tstate[at * kScales + j] != 0 || *(volatile int32_t *)(p.found + at) > j)) {
        if (corner_lane) rmath::corner_advance(cq);
        continue;
      }
      // per-(chart, scale) constants, lane-parallel: lanes 0-19 the local-AABB
      // pieces, lanes 20-21 the OBB line terms, lanes 24-31 the corners
      if (lane < 2 * rmath::kK) {
        const int ax = lane >= rmath::kK, i = lane - ax * rmath::kK;
        rmath::setup_piece(ax ? a1 : a0, i, pb0, pb1, (uint32_t)k, plq, phq);
        rmath::setup_cross(ax ? a1 : a0, i, ce0, ce1, (uint32_t)(ax ? sh.Hq : sh.Wq), (uint32_t)k, cb0, cb1);
      } else if (lane < 2 * rmath::kK + 2) {
        const int ax = lane - 2 * rmath::kK;
        rmath::setup_obb_k(ax ? a1 : a0, ax, sh.Wq, sh.Hq, k, C, S, sh.u0, sh.u1, sh.v0, sh.v1);
      } else if (corner_lane) {
        const int ax = (lane - 24) >> 2;
        rmath::corner_store(cq, lane - 24, ax ? a1 : a0, (ax ? sh.Hq : sh.Wq) * k);
        rmath::corner_advance(cq);
      }
      __syncwarp();
      const int64_t js = (int64_t)j * N + s;
      const int32_t cstart = p.colstart[js];
      const int64_t cbase = p.abase[region(at, j, 0)], rbase = p.abase[region(at, j, 1)];
      const int32_t maxbot = warp_axis(a0, g, p.colpool + cbase + cstart);
      {  // each column word's chart, so a staged run of words knows its owners
        int32_t *own = p.colown + cbase + cstart;
        for (int c = lane; c < a0.len + 2 * g; c += 32) own[c] = s - cb;
      }
      warp_axis(a1, g, p.pool + rbase + p.rowstart[js]);
      if (lane == 0) {
        p.meta[js * 4 + 3] = maxbot;  // w', h' and the column start come from the layout
        atomicAdd(&cta_words[0], (unsigned long long)(a0.len + a1.len + 4 * g));
        atomicAdd(&cta_words[1], (unsigned long long)(a0.len + 2 * g));
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 && cta_words[threadIdx.x]) atomicAdd(p.raster_words + threadIdx.x, cta_words[threadIdx.x]);
}

// Exclusive block scan of the pair (x, y); every thread also gets the
// totals.  part: [66] shared; the caller passes a barrier before the next
// call reuses it.
__device__ __forceinline__ void block_scan2(int64_t &x, int64_t &y, int64_t &tx, int64_t &ty,
                                            int64_t *part) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  int64_t ix = x, iy = y;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t ux = __shfl_up_sync(0xffffffffu, ix, o), uy = __shfl_up_sync(0xffffffffu, iy, o);
    if (lane >= o) { ix += ux; iy += uy; }
  }
  if (lane == 31) { part[w] = ix; part[32 + w] = iy; }
  __syncthreads();
  if (w == 0) {
    const int64_t px = lane < nw ? part[lane] : 0, py = lane < nw ? part[32 + lane] : 0;
    int64_t qx = px, qy = py;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t ux = __shfl_up_sync(0xffffffffu, qx, o), uy = __shfl_up_sync(0xffffffffu, qy, o);
      if (lane >= o) { qx += ux; qy += uy; }
    }
    part[lane] = qx - px;
    part[32 + lane] = qy - py;
    if (lane == 31) { part[64] = qx; part[65] = qy; }
  }
  __syncthreads();
  x = part[w] + ix - x;
  y = part[32 + w] + iy - y;
  tx = part[64];
  ty = part[65];
}

// Pool layouts.  For each (atlas, candidate): the padded column count
// w'(k) = ceil(Wq k / 2^18) + 2g and row count h'(k) of every chart,
// exclusive-scanned in sorted order, so any run of consecutive charts has
// its columns in one contiguous range; the sizes and column starts also go
// to the meta record.  One CTA per (atlas, candidate); each thread sums a
// run of consecutive charts, then a block scan.
__global__ void __launch_bounds__(1024) layout_kernel(const Pack *__restrict__ pp) {
  __shared__ int64_t part[66];
  const Pack &p = *pp;
  const int tid = threadIdx.x;
  const int64_t N = p.N;
  const int g2 = 2 * p.g;
  for (int64_t item = blockIdx.x; item < (int64_t)p.A * kScales; item += gridDim.x) {
    const int at = (int)(item / kScales), j = (int)(item % kScales);
    // candidates above the area bound's top are never evaluated
    if (j > p.jtop[at]) continue;
    const int n = p.atl[at].n, cb = p.atl[at].cb;
    const int64_t k = 16 * (j + 1);
    const int P = (n + 1023) >> 10;
    const int s0 = min(n, tid * P), s1 = min(n, s0 + P);
    int64_t sc = 0, sr = 0;
    for (int s = s0; s < s1; ++s) {
      sc += ((p.wq[cb + s] * k + kFix - 1) >> 18) + g2;
      sr += ((p.hq[cb + s] * k + kFix - 1) >> 18) + g2;
    }
    int64_t tx = 0, ty = 0;
    block_scan2(sc, sr, tx, ty, part);
    const bool meta = j <= p.jtop[at];  // candidates the search may evaluate
    for (int s = s0; s < s1; ++s) {
      const int64_t js = (int64_t)j * N + cb + s;
      const int32_t wp = (int32_t)(((p.wq[cb + s] * k + kFix - 1) >> 18) + g2);
      const int32_t hp = (int32_t)(((p.hq[cb + s] * k + kFix - 1) >> 18) + g2);
      p.colstart[js] = (int32_t)sc;
      p.rowstart[js] = (int32_t)sr;
      // w', h' and the column start of every chart are known before any
      // envelope is drawn (the row loop folds rows of charts not yet drawn)
      if (meta) *reinterpret_cast<int4 *>(p.meta + js * 4) = make_int4(wp, hp, (int32_t)sc, 0);
      sc += wp;
      sr += hp;
    }
    if (tid == 0) {
      // regions are whole 16-byte segments, so staged int4 loads stay aligned
      const int64_t c4 = (tx + 3) & ~3LL, r4 = (ty + 3) & ~3LL;
      p.atot[region(at, j, 0)] = c4;
      p.atot[region(at, j, 1)] = r4;
      const int r = p.jtop[at] - j;  // rank below the atlas's top candidate
      if (r >= 0) {
        atomicAdd(p.jtot + 2 * r, (unsigned long long)c4);
        atomicAdd(p.jtot + 2 * r + 1, (unsigned long long)r4);
      }
    }
    __syncthreads();
  }
}

// Region bases.  Candidates of one wave share the pools (the candidates of
// the next wave reuse them).  A wave holds the ranks r = wF .. wF + F - 1
// below each atlas's top candidate; within a wave the lower ranks come
// first, within a rank the atlases in batch order.  An atlas whose region
// runs past a pool's end is marked out of memory (and never rasterized).
__global__ void __launch_bounds__(1024) bases_kernel(const Pack *__restrict__ pp) {
  __shared__ int64_t part[66];
  __shared__ int64_t carry[2];
  const Pack &p = *pp;
  const int tid = threadIdx.x, r = blockIdx.x;
  const int r0 = r - r % p.F;  // first rank of this wave
  int64_t offc = 0, offr = 0;
  for (int rr = r0; rr < r; ++rr) {
    offc += (int64_t)p.jtot[2 * rr];
    offr += (int64_t)p.jtot[2 * rr + 1];
  }
  if (tid == 0) { carry[0] = offc; carry[1] = offr; }
  __syncthreads();
  for (int base = 0; base < p.A; base += 1024) {
    const int at = base + tid;
    const int j = at < p.A ? p.jtop[at] - r : -1;
    const int64_t vc = j >= 0 ? p.atot[region(at, j, 0)] : 0, vr = j >= 0 ? p.atot[region(at, j, 1)] : 0;
    int64_t ec = vc, er = vr, tx = 0, ty = 0;
    block_scan2(ec, er, tx, ty, part);
    if (j >= 0) {
      const int64_t bc = carry[0] + ec, br = carry[1] + er;
      p.abase[region(at, j, 0)] = bc;
      p.abase[region(at, j, 1)] = br;
      if (bc + vc > p.col_cap || br + vr > p.row_cap) atomicOr(p.err + at, kErrPool);
    }
    __syncthreads();
    if (tid == 0) { carry[0] += tx; carry[1] += ty; }
    __syncthreads();
  }
}

// Wave plan: the atlases still searching (no success yet, no error, and
// candidates left for this wave), in batch order, and a flat list of their
// charts in chunk q.
__global__ void __launch_bounds__(1024) plan_kernel(const Pack *__restrict__ pp, int q) {
  __shared__ int64_t part[66];
  __shared__ int64_t carry[2];
  const Pack &p = *pp;
  const int wave = *(volatile const int32_t *)p.cur_wave;
  const int tid = threadIdx.x;
  if (tid == 0) { carry[0] = 0; carry[1] = 0; }
  __syncthreads();
  for (int base = 0; base < p.A; base += 1024) {
    const int at = base + tid;
    // candidates below the atlas's moot bound (`found`: set by successes,
    // Sec. 4.4's choice) can no longer win; the atlas takes part while the
    // wave holds a candidate at or above it
    const int top = at < p.A ? p.jtop[at] - wave * p.F : -1;
    const int fnd = at < p.A ? *(volatile int32_t *)(p.found + at) : 0;
    bool live = at < p.A && *(volatile uint32_t *)(p.err + at) == 0 && top >= 0 && top >= fnd;
    if (live && q > 0 && !(p.flags & TABI_F_EVAL_ALL)) {
      // a later chunk only for atlases with a candidate of the wave still running
      const WaveRange wr = wave_range(p.jtop[at], wave, p.F);
      bool running = false;
      for (int j = max(wr.lo, fnd); j <= wr.hi && !running; ++j) running = p.tstate[at * kScales + j] == 0;
      live = running;
    }
    const int n = live ? p.atl[at].n : 0;
    int64_t ea = live ? 1 : 0, ec = live ? chunk_end(n, q, p.Q) - (q ? chunk_end(n, q - 1, p.Q) : 0) : 0;
    int64_t tx = 0, ty = 0;
    block_scan2(ea, ec, tx, ty, part);
    if (live) {
      p.act_atl[carry[0] + ea] = at;
      p.act_pre[carry[0] + ea] = (int32_t)(carry[1] + ec);
    }
    __syncthreads();
    if (tid == 0) { carry[0] += tx; carry[1] += ty; }
    __syncthreads();
  }
  if (tid == 0) {
    p.act_info[0] = (int32_t)carry[0];
    p.act_info[1] = (int32_t)carry[1];
    p.counter[wave * kChunkSlots + q] = 0;
  }
}

__global__ void __launch_bounds__(256) plan_fill_kernel(const Pack *__restrict__ pp, int q) {
  const Pack &p = *pp;
  const int na = p.act_info[0];
  for (int i = blockIdx.x; i < na; i += gridDim.x) {
    const int at = p.act_atl[i], pre = p.act_pre[i];
    const int n = p.atl[at].n, cb = p.atl[at].cb, jt = p.jtop[at];
    const int c0 = q ? chunk_end(n, q - 1, p.Q) : 0, c1 = chunk_end(n, q, p.Q);
    for (int t = threadIdx.x; t < c1 - c0; t += blockDim.x) {
      const int c = c0 + t;
      p.act_ext[pre + t] = make_int4(cb + c, at, jt, (int32_t)((uint32_t)cb | (c == n - 1 ? 1u << 31 : 0u)));
    }
  }
}

// ---------------------------------------------------------------------------
// horizontal compactor (Sec. 4.1.2, App. A interlock)
// ---------------------------------------------------------------------------
// One group of G lanes per (scale, sorted pair (s, s+1)), A = s left of
// B = s+1, top-aligned:  d = w'_A - max_r (R'_A(r) - L'_B(r));  B may move
// up relative to A iff every row of B stays right of all rows of A above
// it; A may move up relative to B iff every row of A stays left of all rows
// of B above it.  Groups narrower than a warp keep more pairs' chains of
// dependent loads in flight (the kernel waits on memory, not on issue).
// Items are the charts c of chunk q: the pair (c - 1, c) (both charts are
// drawn by the end of the chunk), and the atlas's last chart's empty pair.
template <int G>
__global__ void __launch_bounds__(256, 6) hcompact_kernel(const Pack *__restrict__ pp, int q, int nj) {
  const Pack &p = *pp;
  const int wave = *(volatile const int32_t *)p.cur_wave;
  const int lane = threadIdx.x & (G - 1);
  const unsigned gm = group_mask<G>();
  const int64_t total = p.act_info[1];
  const int64_t items = total * nj;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const int64_t N = p.N;
  const bool all = q == 0 || (p.flags & TABI_F_EVAL_ALL);
  // the chain of dependent loads per item is kept short: the chart, its
  // atlas and top candidate in one record; the pair's sizes and row
  // starts issued together with the candidate's state
  for (int64_t it = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G; it < items; it += ngroups) {
    const int4 e = p.act_ext[it % total];
    const int c = e.x, at = e.y;
    const WaveRange wr = wave_range(e.z, wave, nj);
    const int j = wr.hi - (int)(it / total);
    if (j < wr.lo) continue;  // this atlas has fewer candidates left than the wave
    const bool first = c == (e.w & 0x7fffffff);
    PairRows pr{};
    if (!first) pr = pair_rows(p, at, j, c - 1);
    if (!all && (p.tstate[at * kScales + j] || *(volatile int32_t *)(p.found + at) > j))
      continue;  // the candidate has finished, or a larger one has succeeded
    if (e.w < 0 && lane == 0) {  // no right neighbour
      p.dnext[(int64_t)j * N + c] = 0;
      p.pflags[(int64_t)j * N + c] = 0;
    }
    if (first) continue;
    compact_rows<G>(p, pr, lane, gm);
  }
}

// After a wave: the next wave index, and whether any atlas can still search
// in it (no error, and the next wave's top candidate exists and is not
// below the atlas's moot bound); inside a captured graph that decides
// whether the wave loop runs again.
__global__ void __launch_bounds__(1024) wave_end_kernel(const Pack *__restrict__ pp, cudaGraphConditionalHandle h,
                                                        int in_graph) {
  __shared__ int any;
  const Pack &p = *pp;
  const int w = *(volatile const int32_t *)p.cur_wave + 1;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int at = threadIdx.x; at < p.A; at += blockDim.x)
    if (p.err[at] == 0 && p.jtop[at] - w * p.F >= max(p.found[at], 0)) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    *p.cur_wave = w;
    if (in_graph) cudaGraphSetConditional(h, (any && w < p.nwaves) ? 1u : 0u);
  }
}

}  // namespace

void launch_layout(const Pack *dp, const Launch &L, cudaStream_t st) {
  layout_kernel<<<L.sms * 2, 1024, 0, st>>>(dp);
  bases_kernel<<<kScales, 1024, 0, st>>>(dp);
}

void launch_plan(const Pack *dp, const Launch &L, int q, cudaStream_t st) {
  plan_kernel<<<1, 1024, 0, st>>>(dp, q);
  plan_fill_kernel<<<L.sms * 2, 256, 0, st>>>(dp, q);
}

void launch_raster(const Pack *dp, const Launch &L, int q, int F, cudaStream_t st) {
  // persistent: the three 256-thread CTAs that fit a multiprocessor at 80 registers
  raster_kernel<<<L.sms * 3, kRasterThreads, 0, st>>>(dp, q, F);
}

constexpr int kHcGroup = 16;
void launch_hcompact(const Pack *dp, const Launch &L, int q, int F, cudaStream_t st) {
  // persistent: six 256-thread CTAs per multiprocessor (40 registers with
  // the loads hoisted; eight CTAs at 32 registers spill)
  hcompact_kernel<kHcGroup><<<L.sms * 6, 256, 0, st>>>(dp, q, F);
}

void launch_wave_end(const Pack *dp, cudaGraphConditionalHandle h, bool in_graph, cudaStream_t st) {
  wave_end_kernel<<<1, 1024, 0, st>>>(dp, h, in_graph ? 1 : 0);
}

}  // namespace tabi
