// The prefix-sum tail of Sec. 4.4 between its two row-loop passes.
//
// When a wave's last chunk is done, every (atlas, candidate S) task that
// switched to the tail has folded its remaining charts at S: the prefix of
// the offsets cut modulo W' into rows, recorded in the tasks' place records
// (tail row per chart, row length at each row's first chart).  Those rows
// may overflow W'.  The kernels here choose the intermediate scale k': the
// largest of S - 14 .. S (one step of the candidate grid) at which every
// row, re-laid from its near end with the charts drawn at k', fits W';
// then redraw the tail charts at k' into the task's own envelope region (at
// k' <= S a chart's padded sizes are no larger than at S, so it fits the
// place it had) and compact them.  The row loop's second pass then drops
// the rows onto the frontline -- or, where no such k' exists, folds the
// remaining charts row by row as before the switch.
//
//   tail_plan     the tail tasks of the wave;
//   tail_trial    a warp per (task, row, trial scale): the row's extent at
//                 that scale, its compacting distances drawn on the fly
//                 (warp_pair_reach), against W' -- the trial scales in four
//                 phases from the top (S .. S - 3, S - 4 .. S - 7, ...);
//   tail_pick     a thread per task, after each phase: the largest scale of
//                 the phase at which every row fit settles the task (every
//                 larger scale has failed); a task none fit goes on to the
//                 next phase, and after the last one to the row-by-row
//                 fallback;
//   tail_raster   a warp per (task, tail chart): its envelope at k';
//   tail_compact  a group of 16 lanes per (task, tail pair): distances and
//                 interlock flags at k'.
#include "raster_dev.cuh"

namespace tabi {
namespace {

constexpr int kTailThreads = 256;
constexpr int kTailWarps = kTailThreads / 32;

// The parked state of a task (its row-loop slot in the wave).
__device__ __forceinline__ int32_t *task_state(const Pack &p, int at, int j, int wave) {
  const int64_t slot = (int64_t)at * p.F + (wave_range(p.jtop[at], wave, p.F).hi - j);
  return p.ctl_save + slot * kCtlSave;
}

// Trial scale i (0..14) of a round: lo + floor((i + 1)(hi - lo) / 16).
__device__ __forceinline__ int32_t trial_scale(int32_t lo, int32_t hi, int i) {
  return lo + (int32_t)(((int64_t)(i + 1) * (hi - lo)) / 16);
}

// The trial scales of phase ph: indices 14 - 4 ph down to 11 - 4 ph (and
// not below 0).
constexpr int kTailPhases = 4;
constexpr int kPhaseScales = 4;
__device__ __forceinline__ int phase_top(int ph) { return 14 - kPhaseScales * ph; }

// Round r of the wave's tail: per atlas, the largest 2^r parked tasks (all
// of them in the last round) that can still win -- a parked candidate below
// the atlas's moot bound is finished as moot.  Only the largest successful
// candidate can win once the tail's downscale is bounded by a grid step (a
// smaller candidate's area-weighted scale stays below the larger one's), so
// the tails are searched and pushed from the top down and the ones a
// success makes moot are never searched.
__global__ void __launch_bounds__(1024) tail_plan_kernel(const Pack *__restrict__ pp, int round, int rounds) {
  __shared__ int32_t count;
  const Pack &p = *pp;
  const int wave = *(volatile const int32_t *)p.cur_wave;
  if (threadIdx.x == 0) count = 0;
  __syncthreads();
  const bool eval_all = (p.flags & TABI_F_EVAL_ALL) != 0;
  const int quota = round + 1 >= rounds ? kScales : 1 << round;
  for (int at = threadIdx.x; at < p.A; at += blockDim.x) {
    const WaveRange wr = wave_range(p.jtop[at], wave, p.F);
    int taken = 0;
    for (int j = wr.hi; j >= wr.lo && j >= 0; --j) {
      if (p.tstate[at * kScales + j] != kTaskTailSearch) continue;
      int32_t *cs = task_state(p, at, j, wave);
      if (!eval_all && *(volatile int32_t *)(p.found + at) > j) {  // moot: a larger candidate succeeded
        ScaleOut &so = p.scale_out[at * kScales + j];
        so.success = 0;
        so.rows = cs[kCsHeadRows];
        so.placed = cs[kCsC0];
        so.score = cs[kCsCommitted];
        so.knee_rows = cs[8];
        so.knees = cs[9];
        so.tail_rows = 0;
        so.tail_k = 0;
        so.tail_start = p.atl[at].n;
        so.evaluated = 2;
        p.tstate[at * kScales + j] = kTaskDone;
        continue;
      }
      if (taken == quota) continue;
      ++taken;
      const int32_t S = 16 * (j + 1);
      cs[kCsLo] = S - 15;  // the trial scales S - 14 .. S
      cs[kCsHi] = S + 1;
      cs[kCsMask] = 0;
      cs[kCsRound] = round;
      cs[kCsKt] = 0;
      p.ttask[atomicAdd(&count, 1)] = make_int4(at, j, 0, cs[kCsC0]);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *p.tcount = count;
    p.counter[wave * kChunkSlots + p.Q] = 0;  // the push pass's task counter
  }
}

// The compacting offsets of a phase (Algorithm 4's x_{t+1} - x_t before the
// clamp, w'_t - d_t = min(w'_t, reach)) of every tail pair (u, u + 1) in one
// row, at the phase's four trial scales: a group of G lanes per (pair,
// scale) draws the two charts' rows at that scale on the fly
// (group_pair_reach).  They go to the tail charts' place records, whose x
// and y are free until the push pass: four int16 (|offset| <= 8192), the
// phase's scale i in slot phase_top - i.
__device__ __forceinline__ int16_t *offset_slot(int4 *place, int u, int slot) {
  return reinterpret_cast<int16_t *>(&place[u].x) + slot;
}

template <int G>
__global__ void __launch_bounds__(kTailThreads) tail_offsets_kernel(const Pack *__restrict__ pp, int phase) {
  constexpr int PG = 32 / G;
  __shared__ rmath::AxisK axk[kTailWarps][2 * PG];
  const Pack &p = *pp;
  if (!(p.flags & TABI_F_HC)) return;  // no compaction: the offsets are the widths
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, grp = lane / G, glane = lane & (G - 1);
  const unsigned gm = group_mask<G>();
  const int g = p.g;
  rmath::AxisK *a = axk[wib];
  const int64_t gw = (int64_t)blockIdx.x * kTailWarps + wib, nw = (int64_t)gridDim.x * kTailWarps;
  const int wave = *(volatile const int32_t *)p.cur_wave;
  const int ntask = *p.tcount;
  for (int ti = 0; ti < ntask; ++ti) {
    const int4 tt = p.ttask[ti];
    const int at = tt.x, j = tt.y, c0 = tt.w;
    if (p.tstate[at * kScales + j] != kTaskTailSearch) continue;
    const int32_t *cs = task_state(p, at, j, wave);
    const int32_t lo = cs[kCsLo], hi = cs[kCsHi];
    const AtlasDesc &ad = p.atl[at];
    const int cb = ad.cb, n = ad.n;
    int4 *place = p.place + (int64_t)j * p.N + cb;
    // items (pair u, scale of the phase), the groups of a warp take PG
    // consecutive ones
    const int64_t items = (int64_t)(n - 1 - c0) * kPhaseScales;
    for (int64_t base = gw * PG; base < items; base += nw * PG) {
      const int64_t it = base + grp;
      int u = 0, slot = 0;
      int32_t k = 0;
      bool pair = false;
      if (it < items) {
        u = c0 + (int)(it / kPhaseScales);
        slot = (int)(it % kPhaseScales);
        const int i = phase_top(phase) - slot;
        if (i >= 0) {
          k = trial_scale(lo, hi, i);
          pair = k > lo && k < hi && !(place[u + 1].w & kTailFirst);
        }
      }
      if (pair) {
        group_setup_rows<G>(p, p.shape[cb + u], k, a[2 * grp], glane);
        group_setup_rows<G>(p, p.shape[cb + u + 1], k, a[2 * grp + 1], glane);
      }
      __syncwarp();
      if (pair) {
        const int32_t M = group_pair_reach<G>(a[2 * grp], a[2 * grp + 1], g, glane, gm);
        const int32_t w = (int32_t)((p.wq[cb + u] * (int64_t)k + kFix - 1) >> 18) + 2 * g;
        if (glane == 0) *offset_slot(place, u, slot) = (int16_t)(w - M > 0 ? M : w);
      }
      __syncwarp();  // the buffers are redrawn next step
    }
  }
}

// Whether the tail row starting at sorted chart s0 (len charts) fits W' when
// laid from its near end at scale k, the phase's slot `slot`: Algorithm 4's
// recurrence x_{t+1} = x_t + o_t, with compaction never left of the right
// edge of chart t-1, from the stored offsets; a warp loads 32 charts at a
// time and walks them.
__device__ bool row_fits(const Pack &p, const int4 *place, int cb, int s0, int len, int64_t k, int Wp, int slot,
                         const volatile int32_t *mask, int bit) {
  const bool hc = (p.flags & TABI_F_HC) != 0;
  const int g = p.g;
  const int lane = threadIdx.x & 31;
  int64_t x = 0, xprev = 0, wprev = 0, ext = 0;
  for (int t = 0; t < len; t += 32) {
    // another row has already failed at this scale: the outcome is known
    if (__shfl_sync(0xffffffffu, lane == 0 ? (*mask >> bit) & 1 : 0, 0)) return true;
    const int u = s0 + t + lane;
    int64_t w = 0, o = 0;
    if (t + lane < len) {
      w = ((p.wq[cb + u] * k + kFix - 1) >> 18) + 2 * g;
      o = (hc && t + lane + 1 < len) ? (int64_t)*reinterpret_cast<const int16_t *>(
                                           reinterpret_cast<const int16_t *>(&place[u].x) + slot)
                                     : w;
    }
    const int cnt = min(32, len - t);
    for (int q = 0; q < cnt; ++q) {
      const int64_t oq = __shfl_sync(0xffffffffu, o, q), wq = __shfl_sync(0xffffffffu, w, q);
      ext = ext > x + wq ? ext : x + wq;
      if (ext > Wp) return false;
      int64_t nx = x + oq;
      if (hc && t + q >= 1 && nx < xprev + wprev) nx = xprev + wprev;
      xprev = x;
      wprev = wq;
      x = nx;
    }
  }
  return true;
}

__global__ void __launch_bounds__(kTailThreads) tail_trial_kernel(const Pack *__restrict__ pp, int phase) {
  const Pack &p = *pp;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * kTailWarps + wib, nw = (int64_t)gridDim.x * kTailWarps;
  const int wave = *(volatile const int32_t *)p.cur_wave;
  const int ntask = *p.tcount;
  for (int ti = 0; ti < ntask; ++ti) {
    const int4 tt = p.ttask[ti];
    const int at = tt.x, j = tt.y, c0 = tt.w;
    if (p.tstate[at * kScales + j] != kTaskTailSearch) continue;
    const int32_t *cs = task_state(p, at, j, wave);
    const int32_t lo = cs[kCsLo], hi = cs[kCsHi];
    const AtlasDesc &ad = p.atl[at];
    const int cb = ad.cb, n = ad.n, Wp = ad.W + 2 * p.g;
    const int4 *place = p.place + (int64_t)j * p.N + cb;
    const int64_t items = (int64_t)(n - c0) * kPhaseScales;
    for (int64_t it = gw; it < items; it += nw) {
      const int s = c0 + (int)(it / kPhaseScales), slot = (int)(it % kPhaseScales), i = phase_top(phase) - slot;
      if (i < 0) continue;
      const int32_t w = place[s].w;
      if (!(w & kTailFirst)) continue;  // rows are tried from their first chart
      const int32_t k = trial_scale(lo, hi, i);
      if (k <= lo || k >= hi) continue;
      // a scale at which some row has failed is decided: its other rows are
      // skipped (the mask only gathers failures, so the outcome is the same)
      const volatile int32_t *mask = cs + kCsMask;
      if ((*mask >> i) & 1) continue;
      if (!row_fits(p, place, cb, s, w & ~kTailFirst, k, Wp, slot, mask, i) && lane == 0)
        atomicOr((unsigned *)(cs + kCsMask), 1u << i);
    }
  }
}

// The outcome of a phase per task (a thread each): k' is the largest trial
// scale of the phase at which every row fit (its bit in the mask is clear;
// every scale of the earlier phases failed); a task without one stays in
// the search for the next phase, or after the last takes k' = 0.  A
// settled task goes on to the push pass.
__global__ void tail_pick_kernel(const Pack *__restrict__ pp, int phase) {
  const Pack &p = *pp;
  const int wave = *(volatile const int32_t *)p.cur_wave;
  const int ntask = *p.tcount;
  for (int ti = blockIdx.x * blockDim.x + threadIdx.x; ti < ntask; ti += gridDim.x * blockDim.x) {
    const int4 tt = p.ttask[ti];
    const int at = tt.x, j = tt.y;
    if (p.tstate[at * kScales + j] != kTaskTailSearch) continue;
    int32_t *cs = task_state(p, at, j, wave);
    const int32_t lo = cs[kCsLo], hi = cs[kCsHi];
    const uint32_t mask = (uint32_t)cs[kCsMask];
    int32_t best = 0;
    for (int i = max(0, phase_top(phase) - kPhaseScales + 1); i <= phase_top(phase); ++i) {
      const int32_t k = trial_scale(lo, hi, i);
      if (k > lo && k < hi && !((mask >> i) & 1u) && k > best) best = k;
    }
    if (best == 0 && phase + 1 < kTailPhases) continue;  // the next phase's scales
    cs[kCsKt] = best;
    cs[kCsMask] = 0;
    p.tstate[at * kScales + j] = kTaskTailPush;
  }
}

// The tail charts at k', in the place their envelopes had at S: columns
// (and their owners), rows, and the padded sizes and deepest bottom.
__global__ void __launch_bounds__(kTailThreads) tail_raster_kernel(const Pack *__restrict__ pp) {
  __shared__ rmath::AxisK axk[kTailWarps][2];
  const Pack &p = *pp;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * kTailWarps + wib, nw = (int64_t)gridDim.x * kTailWarps;
  const int wave = *(volatile const int32_t *)p.cur_wave;
  const int ntask = *p.tcount;
  const int g = p.g;
  for (int ti = 0; ti < ntask; ++ti) {
    const int4 tt = p.ttask[ti];
    const int at = tt.x, j = tt.y, c0 = tt.w;
    if (p.tstate[at * kScales + j] != kTaskTailPush) continue;
    const int32_t kt = task_state(p, at, j, wave)[kCsKt];
    const AtlasDesc &ad = p.atl[at];
    const int cb = ad.cb, n = ad.n;
    // the trial offsets leave the tail records' x and y as they were (zero)
    int2 *xy = reinterpret_cast<int2 *>(p.place + (int64_t)j * p.N + cb);
    for (int64_t s = c0 + gw * 32 + lane; s < n; s += nw * 32) xy[2 * s] = make_int2(0, 0);
    if (kt == 0) continue;  // no tail scale: the rows go on at S
    const int64_t cbase = p.abase[region(at, j, 0)], rbase = p.abase[region(at, j, 1)];
    for (int64_t s = c0 + gw; s < n; s += nw) {
      const int64_t js = (int64_t)j * p.N + cb + s;
      rmath::AxisK &a0 = axk[wib][0], &a1 = axk[wib][1];
      setup_at_k(p, p.shape[cb + s], kt, &a0, &a1);
      const int32_t cstart = p.colstart[js];
      const int32_t wold = p.meta[js * 4];  // padded width at S: the words this chart owns
      __syncwarp();
      const int32_t maxbot = warp_axis(a0, g, p.colpool + cbase + cstart);
      int32_t *own = p.colown + cbase + cstart;
      // the words past the narrower envelope belong to no chart (-1): the row
      // loop's commit skips them
      for (int c = lane; c < wold; c += 32) own[c] = c < a0.len + 2 * g ? (int32_t)s : -1;
      warp_axis(a1, g, p.pool + rbase + p.rowstart[js]);
      if (lane == 0)
        *reinterpret_cast<int4 *>(p.meta + js * 4) = make_int4(a0.len + 2 * g, a1.len + 2 * g, cstart, maxbot);
      __syncwarp();
    }
  }
}

constexpr int kCompactGroup = 16;

__global__ void __launch_bounds__(256) tail_compact_kernel(const Pack *__restrict__ pp) {
  const Pack &p = *pp;
  constexpr int G = kCompactGroup;
  const int lane = threadIdx.x & (G - 1);
  const unsigned gm = group_mask<G>();
  const int64_t gg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t ng = ((int64_t)gridDim.x * blockDim.x) / G;
  const int ntask = *p.tcount;
  for (int ti = 0; ti < ntask; ++ti) {
    const int4 tt = p.ttask[ti];
    const int at = tt.x, j = tt.y, c0 = tt.w;
    if (p.tstate[at * kScales + j] != kTaskTailPush) continue;
    if (task_state(p, at, j, *(volatile const int32_t *)p.cur_wave)[kCsKt] == 0) continue;
    const int cb = p.atl[at].cb, n = p.atl[at].n;
    for (int64_t s = c0 + gg; s + 1 < n; s += ng) compact_pair<G>(p, at, j, cb + (int)s, lane, gm);
  }
}

}  // namespace

int tail_rounds(int F) {
  int r = 1;
  while ((1 << r) - 1 < F && r < 7) ++r;  // quotas 1, 2, 4, ... then the rest
  return r;
}

void launch_tail_round(const Pack *dp, const Launch &L, int F, int round, cudaStream_t st) {
  tail_plan_kernel<<<1, 1024, 0, st>>>(dp, round, tail_rounds(F));
  for (int ph = 0; ph < kTailPhases; ++ph) {
    // groups of 8 lanes per pair while the gutter dilation (2g) stays inside
    // one chunk of 8 rows, else a warp per pair
    if (L.gutter <= 3) tail_offsets_kernel<8><<<L.sms * 4, kTailThreads, 0, st>>>(dp, ph);
    else tail_offsets_kernel<32><<<L.sms * 4, kTailThreads, 0, st>>>(dp, ph);
    tail_trial_kernel<<<L.sms * 4, kTailThreads, 0, st>>>(dp, ph);
    tail_pick_kernel<<<L.sms, 128, 0, st>>>(dp, ph);
  }
  tail_raster_kernel<<<L.sms * 3, kTailThreads, 0, st>>>(dp);
  tail_compact_kernel<<<L.sms * 8, 256, 0, st>>>(dp);
}

}  // namespace tabi
