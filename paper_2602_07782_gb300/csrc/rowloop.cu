// Row loop of one (atlas, candidate scale): Algorithm 5 (with Algorithms 2,
// 3, 4 and the hierarchical selection of Sec. 4.2).  The kernel is
// persistent, one CTA per multiprocessor; each CTA takes (atlas, candidate)
// tasks of the current wave from a device counter.
//
// Lazy evaluation: a wave draws the envelopes chunk by chunk of the sorted
// charts (e.g. first 1/8, next 1/8, 1/4, 1/2; see chunk_end), and after
// each chunk the row loop
// of every candidate still running commits the rows it can decide with the
// charts drawn so far, then parks its frontline and row state until the
// next chunk.  A candidate that fails (most candidates above the answer
// fail after a fraction of their charts) gets no further envelopes.  A row
// is decided only if the first chart that does not fit in any fold is drawn,
// so every decision is the one the whole-atlas loop would make.
//
// Shared memory holds the committed frontline (one int per padded atlas
// column) and the per-row working set.  A row proceeds in barrier-separated
// phases:
//   A  knee refresh (Algorithm 3) and the concavity's current maximum;
//   B  folds (Algorithm 4): warp 0 folds side by side, warp 1 with
//      compaction.  The compacted fold x_{t+1} = max(x_t + w'_t - d_t,
//      x_{t-1} + w'_{t-1}) is a prefix sum wherever the clamp does not
//      bind; a chunk where it binds is redone as a warp scan of 2x2
//      (max,+) matrices applied to the carried state (x_t, x_{t-1}).  A
//      fold from the same first chart serves both the atlas width and the
//      knee width.  The other warps stage the row window (widths, pool
//      offsets, deepest bottoms, interlock bits, heights) into shared
//      memory;
//   D  push: one warp per chart loads its TopEdge once (both orientations)
//      and forms, for every configuration the chart is part of, the maximum
//      of front[x] - TopEdge over its columns;
//   E  per configuration (one warp each) the interlock fixpoint of
//      Algorithm 2 -- the least solution is, per chart, the maximum pushed
//      offset over the charts chained to it, i.e. a forward and a backward
//      segmented max-scan -- and the score.  After the push the frontline's
//      maximum is max(committed maximum, max_c (y_c + max BottomEdge_c)),
//      so configurations never copy the frontline;
//      Two further warps find the knee candidate (App. A) of both
//      atlas-width rows meanwhile;
//   G  selection (Sec. 4.2): every thread derives the same choice from the
//      scores (so no barrier separates it from the commit); thread 0 also
//      advances the row state;
//   H  commit: one warp per chart raises the frontline (shared atomicMax,
//      since compacted neighbours share columns); placements out.
// The progressive area bound after a commit is checked by one thread of
// the next row's staging (phase B), so a row costs four barriers.
//
// Prefix-sum tail (Sec. 4.4): once no knee is live and a row's first
// (tallest) chart is below t_opt of the atlas height (atlases of more than
// hybrid_min charts), phase T switches the task to the tail for good, in
// two passes.  First the fold at the candidate scale: a tail row is the
// same fold, continued from the carried unwrapped prefix (the offsets'
// running sum, clamp included) and cut where the prefix passes the next
// multiple of W' (its last chart may overflow); the row is only recorded
// (its charts' place records carry the tail row and, at its first chart,
// the row length) and nothing is pushed.  Once every chart is folded the
// task parks (state kTaskTailSearch) and the tail kernels search the
// intermediate scale k' (within one grid step below the candidate), redraw
// the tail charts at k' and compact them.  Then the push pass (q = Q, state
// kTaskTailPush): each recorded row is laid from its near end by the same
// fold at k', in the fixed direction pattern left-to-right, right-to-left,
// right-to-left, and phases D, E and H push it as the one configuration of
// the row.  If no k' fitted, the push pass instead folds the remaining
// charts row by row from the switch, exactly as without a tail.
#include "tabi_internal.cuh"

namespace tabi {
namespace {

constexpr int kMaxWarps = 32;
constexpr int32_t kNeg = -(1 << 28);  // max-plus "minus infinity"
constexpr int32_t kI32Min = -0x7fffffff - 1;

struct Ctl {
  int32_t len[4];        // fold variants v = fold * 2 + hc: charts in the row
  int32_t score[8], score_knee[8];
  int32_t row_start, row, committed, fail, prev_ltr, bound_fail, prev_maxlen;
  int32_t knee_valid, knee_ltr, knee_l, knee_r;
  int32_t region_lo, region_hi, knee_max;
  int32_t knee_rows, knees, knee_t[2], stage_lo, stage_hi, abort;
  int32_t t_at, t_j, t_skip;
  int32_t front_sum;     // the committed frontline summed over the padded columns
  // prefix-sum tail (Sec. 4.4): mode (0 off, 1 folding at the candidate
  // scale, 3 pushing at the tail scale, 4 abandoned: no tail scale within a
  // grid step, rows one by one), cut width, unwrapped prefix of the
  // next row's first chart and of the chart before it (have_prev: one
  // exists) with that chart's width, tail rows folded or pushed, first tail
  // chart, rows before it, the tail scale, the pushed row's length
  int32_t tail, tL, tP, tPrev, tWprev, tHave, trows, c0, head_rows, kt, plen;
  int32_t head_p;        // charts surely folded row by row (the progressive bound's share)
  int32_t red[kMaxWarps];
};

// 2x2 max-plus matrix
struct MP {
  int32_t a00, a01, a10, a11;
};
__device__ __forceinline__ int32_t mpadd(int32_t x, int32_t y) {
  const int32_t s = x + y;
  return s < kNeg ? kNeg : s;
}
// (A (x) B)  -- apply B first, then A
__device__ __forceinline__ MP mpmul(const MP &A, const MP &B) {
  MP C;
  C.a00 = max(mpadd(A.a00, B.a00), mpadd(A.a01, B.a10));
  C.a01 = max(mpadd(A.a00, B.a01), mpadd(A.a01, B.a11));
  C.a10 = max(mpadd(A.a10, B.a00), mpadd(A.a11, B.a10));
  C.a11 = max(mpadd(A.a10, B.a01), mpadd(A.a11, B.a11));
  return C;
}
__device__ __forceinline__ MP mpshfl_up(const MP &m, int o) {
  MP r;
  r.a00 = __shfl_up_sync(0xffffffffu, m.a00, o);
  r.a01 = __shfl_up_sync(0xffffffffu, m.a01, o);
  r.a10 = __shfl_up_sync(0xffffffffu, m.a10, o);
  r.a11 = __shfl_up_sync(0xffffffffu, m.a11, o);
  return r;
}

template <int NW>
__device__ __forceinline__ int32_t block_max(int32_t v, Ctl &ctl) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_max(v);
  if (lane == 0) ctl.red[w] = v;
  __syncthreads();
  int32_t r = lane < NW ? ctl.red[lane] : kI32Min;
  r = warp_max(r);
  __syncthreads();
  return r;
}
template <int NW>
__device__ __forceinline__ int32_t block_min(int32_t v, Ctl &ctl) {
  return -block_max<NW>(-v, ctl);
}
template <int NW>
__device__ __forceinline__ int32_t block_sum(int32_t v, Ctl &ctl) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) ctl.red[w] = v;
  __syncthreads();
  int32_t r = lane < NW ? ctl.red[lane] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  __syncthreads();
  return r;
}

// segmented inclusive scan (max) over lanes; `heads` has a bit per lane
// that starts a segment (bit 0 set), each lane's start is its highest head
__device__ __forceinline__ int32_t seg_scan_max(int32_t v, unsigned heads) {
  const int lane = threadIdx.x & 31;
  const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane - o >= start) v = max(v, u);
  }
  return v;
}

// Row capacity: charts in a row start at least 2g + 1 texels apart (each
// padded scanline spans 2g + 1 texels or more), so a row holds at most
// W'/(2g+1) + 1 charts.
__host__ __device__ __forceinline__ int rowloop_maxrow(int W, int g) {
  const int Wp = W + 2 * g;
  return (Wp / (2 * g + 1) + 2 + 3) & ~3;
}

// Persistent: each CTA takes (atlas, candidate) tasks of the wave from a
// device counter, larger candidates of an atlas first.  A task is skipped,
// or abandoned between rows, once a larger candidate of its atlas has
// succeeded (unless every candidate is to be evaluated).
// NT threads per CTA (1024: one CTA per multiprocessor; 512: two).
template <int NT>
__global__ void __launch_bounds__(NT) rowloop_kernel(const Pack *__restrict__ pp, int q, int nj, int smem_words) {
  constexpr int kNT = NT, kNW = NT / 32;
  const Pack &p = *pp;
  const int wave = *(volatile const int32_t *)p.cur_wave;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t flags = p.flags;
  const bool use_hc = flags & TABI_F_HC;
  const bool balance = flags & TABI_F_BALANCE;
  const bool eval_all = flags & TABI_F_EVAL_ALL;
  const bool area_bound = !eval_all && p.prog_bound;  // phase I
  const int vt = use_hc ? 1 : 0;                      // the fold a tail row uses
  const int g = p.g;
  const int64_t N = p.N;
  extern __shared__ int4 sm4[];
  __shared__ Ctl ctl;

  while (true) {
    if (tid == 0) {
      const int t = atomicAdd(p.counter + wave * kChunkSlots + q, 1);
      int at = -1, j = 0, skip = 1;
      const bool push = q >= p.Q;  // the tail's push pass: its tasks come from the tail list
      const int ntask = push ? *(volatile int32_t *)p.tcount : *(volatile int32_t *)p.act_info * nj;
      if (t < ntask) {
        if (push) {
          const int4 tt = p.ttask[t];
          at = tt.x;
          j = tt.y;
          skip = p.tstate[at * kScales + j] != kTaskTailPush;
        } else {
          at = p.act_atl[t / nj];
          const WaveRange wr = wave_range(p.jtop[at], wave, nj);
          j = wr.hi - t % nj;
          skip = j < wr.lo || (q > 0 && p.tstate[at * kScales + j] != kTaskRun);  // outside the wave, or parked
        }
        if (!skip && !eval_all && *(volatile int32_t *)(p.found + at) > j) {
          // a larger candidate has succeeded: this one is moot
          skip = 1;
          if (q > 0) p.scale_out[at * kScales + j].evaluated = 2;  // it ran in an earlier chunk
          p.tstate[at * kScales + j] = kTaskDone;                 // no later chunk runs it
        }
        // the host sizes the CTA for the widest atlas; never overrun it
        const int W = p.atl[at].W;
        if (!skip && smem_words < ((W + 2 * g + 3) & ~3) + 15 * rowloop_maxrow(W, g)) {
          atomicOr(p.err + at, kErrRow);
          skip = 1;
        }
      }
      ctl.t_at = at;
      ctl.t_j = j;
      ctl.t_skip = skip;
    }
    __syncthreads();
    const int at = ctl.t_at, j = ctl.t_j;
    if (at < 0) break;
    if (!ctl.t_skip) {
      const AtlasDesc &ad = p.atl[at];
      const int n = ad.n, cb = ad.cb;
      const int Wp = ad.W + 2 * g, Hp = ad.H + 2 * g;
      const int wp_pad = (Wp + 3) & ~3;
      const int maxrow = rowloop_maxrow(ad.W, g);
      const bool hybrid = p.topt > 0 && n > p.hyb_min;  // Sec. 4.4
      // the column stage takes what is left, up to two atlas widths of words
      // (each staged word costs one word of stage and one of chart index)
      const int room = (smem_words - wp_pad - 15 * maxrow) / 2;
      const int scap = (room < 2 * wp_pad ? (room > 0 ? room : 0) : 2 * wp_pad) & ~3;
      ScaleOut *so = p.scale_out + at * kScales + j;

      uint32_t *stage = reinterpret_cast<uint32_t *>(sm4);  // [scap] the row's column words
      int32_t *front = reinterpret_cast<int32_t *>(sm4) + scap;  // [wp_pad]
      int32_t *posN = front + wp_pad;       // [maxrow] side by side
      int32_t *posH = posN + maxrow;        // [maxrow] compacted
      int32_t *yb = posH + maxrow;          // [8][maxrow]
      int32_t *wps = yb + 8 * maxrow;       // [maxrow] w'
      int32_t *mbot = wps + maxrow;         // [maxrow] max BottomEdge
      int32_t *woff = mbot + maxrow;        // [maxrow] column start in the column pool
      int32_t *pflw = woff + maxrow;        // [maxrow] interlock bits of pair (t, t+1)
      int32_t *hqw = pflw + maxrow;         // [maxrow] unscaled heights
      int32_t *sown = hqw + maxrow;         // [scap] sorted chart index of each staged word

      const int64_t cbase = p.abase[region(at, j, 0)];
      const int64_t ccap = p.col_cap - cbase;  // words readable from the region's start
      const uint32_t *colp = p.colpool + cbase;
      const int32_t *cown = p.colown + cbase;
      const int64_t js = (int64_t)j * N + cb;
      const int32_t *meta = p.meta + js * 4;
      const int32_t *dnext = p.dnext + js;
      const uint8_t *pfl = p.pflags + js;
      const int32_t *hqa = p.hq + cb;
      int4 *place = p.place + js;

      // charts drawn so far (chunks 0..q); rows are decided on them only
      const int avail = q >= p.Q - 1 ? n : chunk_end(n, q, p.Q);
      const int64_t slot = (int64_t)at * p.F + (wave_range(p.jtop[at], wave, nj).hi - j);
      int32_t *fsave = p.front_save + slot * p.wps_stride;
      int32_t *csave = p.ctl_save + slot * kCtlSave;
      if (q == 0) {
        for (int x = tid; x < wp_pad; x += kNT) front[x] = 0;
        if (tid == 0) {
          ctl.row_start = 0; ctl.row = 0; ctl.committed = 0; ctl.prev_ltr = 0;
          ctl.knee_valid = 0; ctl.knee_ltr = 0; ctl.knee_l = 0; ctl.knee_r = 0;
          ctl.knee_rows = 0; ctl.knees = 0;
          ctl.tail = 0; ctl.tL = 1; ctl.tP = 0; ctl.tPrev = 0; ctl.tWprev = 0; ctl.tHave = 0; ctl.trows = 0;
          ctl.c0 = n; ctl.head_rows = 0; ctl.kt = 0;
        }
      } else {  // resume where the previous chunk (or the tail search) stopped
        for (int x = tid; x < wp_pad; x += kNT) front[x] = fsave[x];
        if (tid == 0) {
          ctl.row_start = csave[0]; ctl.row = csave[1]; ctl.committed = csave[2]; ctl.prev_ltr = csave[3];
          ctl.knee_valid = csave[4]; ctl.knee_ltr = csave[5]; ctl.knee_l = csave[6]; ctl.knee_r = csave[7];
          ctl.knee_rows = csave[8]; ctl.knees = csave[9];
          ctl.tail = csave[kCsTail] & 7; ctl.tHave = (csave[kCsTail] >> 3) & 1; ctl.trows = csave[kCsTail] >> 4;
          ctl.tL = csave[11]; ctl.tP = csave[12]; ctl.tPrev = csave[13]; ctl.tWprev = csave[14];
          ctl.c0 = csave[kCsC0]; ctl.head_rows = csave[kCsHeadRows]; ctl.kt = csave[kCsKt];
          if (q >= p.Q) {  // the push pass: the tail rows again from the first, at the tail scale
            ctl.tail = ctl.kt > 0 ? 3 : 4;  // 4: no tail scale fitted, the rows go on one by one
            ctl.row_start = ctl.c0;
            ctl.row = ctl.head_rows;
            ctl.trows = 0;
            ctl.committed = csave[kCsCommitted];
          }
        }
      }
      if (tid == 0)  // charts surely folded row by row at this scale (the rest may end smaller)
        ctl.head_p = area_bound ? head_prefix(hqa, n, 16 * (int64_t)(j + 1), p.topt, ad.H, hybrid) : n;
      {  // the frontline's sum (atlas sides <= 8192: below 2^31), kept up to date by the commits
        int32_t fs = 0;
        if (q > 0 && area_bound)
          for (int x = tid; x < Wp; x += kNT) fs += front[x];
        if (area_bound) fs = block_sum<kNW>(fs, ctl);
        if (tid == 0) { ctl.fail = 0; ctl.bound_fail = 0; ctl.prev_maxlen = 0; ctl.abort = 0; ctl.front_sum = fs; }
      }
      __syncthreads();
      bool deferred = false;
      // progressive area bound: the atlas's totals (per task)
      const unsigned long long tot2 = area_bound ? p.area2[at] : 0, totE = area_bound ? p.ext_sum[at] : 0;

      while (true) {
        const int row_start = ctl.row_start, row = ctl.row;
        if (row_start >= n || ctl.fail) break;
        // row state the selection reads while thread 0 advances it
        const int prev_ltr = ctl.prev_ltr, trows = ctl.trows;

        // ---- T: switch to the prefix-sum tail (Sec. 4.4) ----------------------
        // once no knee is live and the row's first (tallest) chart is shorter
        // than t_opt H at this scale: from here on the charts are folded by
        // the prefix of their offsets with rows cut modulo W' (recorded, not
        // pushed; see the file comment)
        if (hybrid && !ctl.tail && !ctl.knee_valid &&
            1000 * (int64_t)(meta[(int64_t)row_start * 4 + 1] - 2 * g) < (int64_t)p.topt * ad.H) {
          if (tid == 0) {
            ctl.tail = 1; ctl.tL = Wp; ctl.tP = 0; ctl.tHave = 0;
            ctl.c0 = row_start; ctl.head_rows = row;
          }
          __syncthreads();
        }
        if (ctl.tail == 3 && tid == 0) ctl.plen = place[row_start].w & ~kTailFirst;  // a recorded row
        __syncthreads();
        const int tmode = ctl.tail;
        const bool tail = tmode == 1 || tmode == 3;
        // a folded tail row's start in the unwrapped prefix, and its cut width
        const int32_t tB = tmode == 1 ? (ctl.tP / ctl.tL) * ctl.tL : 0, tL = ctl.tL;
        const int32_t plen = ctl.plen;

        // ---- A: knee refresh (Algorithm 3) and the concavity's max -----------
        const bool knee = ctl.knee_valid;
        if (knee) {
          const int L = ctl.knee_l, R = ctl.knee_r;
          if (ctl.knee_ltr) {
            const int32_t cur = front[R];
            int32_t best = L - 1;
            for (int x = L + tid; x < R; x += kNT)
              if (front[x] >= cur) best = max(best, x);
            best = block_max<kNW>(best, ctl);
            if (tid == 0) { ctl.knee_r = best + 1; ctl.region_lo = best + 1; ctl.region_hi = Wp; }
          } else {
            const int32_t cur = front[L - 1];
            int32_t best = R;
            for (int x = L + tid; x < R; x += kNT)
              if (front[x] >= cur) best = min(best, x);
            best = block_min<kNW>(best, ctl);
            if (tid == 0) { ctl.knee_l = best; ctl.region_lo = 0; ctl.region_hi = best; }
          }
          __syncthreads();
          int32_t mx = 0;
          for (int x = ctl.region_lo + tid; x < ctl.region_hi; x += kNT) mx = max(mx, front[x]);
          mx = block_max<kNW>(mx, ctl);
          if (tid == 0) ctl.knee_max = mx;
        }

        // ---- B: folds (Algorithm 4) -------------------------------------------
        if (warp < 2) {
          const int hc = warp;  // warp 0: side by side, warp 1: compacted
          const bool active = tail ? hc == vt : (hc == 0 || use_hc);
          int32_t lenF = 0, lenK = 0;
          if (active) {
            const int32_t foldF = Wp;
            const int32_t foldK = knee ? ctl.region_hi - ctl.region_lo : -1;
            int32_t *pos = hc ? posH : posN;
            // state at the chunk start: x of its first chart, x and right edge
            // of the chart before it (none at the row start)
            int32_t carry_x = 0, carry_xprev = kNeg, carry_re = kNeg, carry_wprev = kNeg;
            if (tmode == 1) {  // continue the prefix, relative to this row's start
              carry_x = ctl.tP - tB;
              if (ctl.tHave) {
                carry_xprev = ctl.tPrev - tB;
                carry_re = carry_xprev + ctl.tWprev;
                carry_wprev = ctl.tWprev;
              }
            }
            bool doneF = false, doneK = !knee;
            // widths and distances of four chunks are loaded together (one
            // memory round trip per 128 charts), then scanned chunk by chunk;
            // a fold stops at the first chart not drawn yet (the row then
            // waits for the next chunk)
            for (int g0 = 0; !(doneF && doneK); g0 += 128) {
              int32_t wq[4], dq[4];
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                const int s = row_start + g0 + 32 * c + lane;
                wq[c] = s < n ? meta[(int64_t)s * 4] : 0;
                dq[c] = (hc && s < avail) ? dnext[s] : 0;
              }
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                if (doneF && doneK) break;
                const int t0 = g0 + 32 * c;
                const int t = t0 + lane;
                const int s = row_start + t;
                const bool valid = s < avail;  // undrawn charts end every fold
                const bool room = t < maxrow;  // the last chunk may run past the row capacity
                const int32_t w = wq[c], d = dq[c];
                const int32_t a = hc ? w - d : w;  // x_{t+1} = x_t + a_t unless the clamp binds
                int32_t incl = a;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                  const int32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                  if (lane >= o) incl += u;
                }
                int32_t xnext = carry_x + incl, xt = xnext - a;
                if (hc) {
                  // clamp: chart t+1 never starts left of chart t-1's right edge
                  int32_t re_prev = __shfl_up_sync(0xffffffffu, xt + w, 1);
                  if (lane == 0) re_prev = carry_re;
                  if (__any_sync(0xffffffffu, valid && xnext < re_prev)) {
                    // the clamp binds in this chunk: (max,+) matrix scan,
                    // state (x_t, x_{t-1}) -> (max(x_t + a_t, x_{t-1} + w_{t-1}), x_t)
                    int32_t wprev = __shfl_up_sync(0xffffffffu, w, 1);
                    if (lane == 0) wprev = carry_wprev;
                    MP m{a, wprev, 0, kNeg};
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                      const MP u = mpshfl_up(m, o);
                      if (lane >= o) m = mpmul(m, u);
                    }
                    xnext = max(mpadd(m.a00, carry_x), mpadd(m.a01, carry_xprev));
                    xt = __shfl_up_sync(0xffffffffu, xnext, 1);
                    if (lane == 0) xt = carry_x;
                  }
                  carry_xprev = __shfl_sync(0xffffffffu, xt, 31);
                  carry_re = __shfl_sync(0xffffffffu, xt + w, 31);
                  carry_wprev = __shfl_sync(0xffffffffu, w, 31);
                }
                carry_x = __shfl_sync(0xffffffffu, xnext, 31);
                // the first chart that does not fit ends the row (a tail row
                // being folded: the first starting at or past the cut; one
                // being pushed: its recorded length)
                const unsigned overF = __ballot_sync(
                    0xffffffffu, !valid || (tmode == 1 ? xt >= tL : tmode == 3 ? t >= plen : xt + w > foldF));
                const unsigned overK = __ballot_sync(0xffffffffu, !valid || xt + w > foldK);
                if (!doneF && overF) { lenF = t0 + __ffs(overF) - 1; doneF = true; }
                else if (!doneF) lenF = t0 + 32;
                if (!doneK && overK) { lenK = t0 + __ffs(overK) - 1; doneK = true; }
                else if (!doneK) lenK = t0 + 32;
                if (valid && room) pos[t] = xt;
                if (t0 + 32 >= maxrow && !(doneF && doneK)) {  // cannot happen: rows hold <= W'/(2g+1) + 1 charts
                  if (lane == 0) atomicOr(p.err + at, kErrRow);
                  doneF = doneK = true;
                }
                if ((doneF && lenF >= maxrow) || (doneK && lenK >= maxrow)) {
                  if (lane == 0) atomicOr(p.err + at, kErrRow);
                  lenF = min(lenF, maxrow - 1);
                  lenK = min(lenK, maxrow - 1);
                }
              }
            }
          }
          if (lane == 0) {
            ctl.len[hc] = active ? lenF : 0;
            ctl.len[2 + hc] = (active && knee) ? lenK : 0;
          }
        } else {
          // meanwhile the other warps stage the row window into shared memory:
          // the column words of the charts from row_start on (contiguous in the
          // column pool; int4 loads from a 16-byte aligned start), and every
          // chart that can be in this row's widths, column starts, deepest
          // bottoms, interlock bits and heights
          const int32_t c4 = meta[(int64_t)row_start * 4 + 2] & ~3;
          const int32_t nw = (int32_t)min((int64_t)scap, ccap - c4) & ~3;
          {
            const int4 *src = reinterpret_cast<const int4 *>(colp + c4);
            const int4 *osrc = reinterpret_cast<const int4 *>(cown + c4);
            int4 *odst = reinterpret_cast<int4 *>(sown);
            for (int q = tid - 64; q < nw / 4; q += kNT - 64) { sm4[q] = src[q]; odst[q] = osrc[q]; }
            if (tid == 64) {
              ctl.stage_lo = c4;
              ctl.stage_hi = c4 + nw;
              // a larger candidate of this atlas has succeeded: this one is moot
              ctl.abort = !eval_all && *(volatile int32_t *)(p.found + at) > j;
              // ---- progressive area bound (exact; an addition to the paper) ----
              // Every later chart is dropped onto the frontline: in column x
              // its cover dilated by g lies inside its padded envelope, at or
              // below front[x], and above the padded atlas bottom Hp (or the
              // candidate fails).  Placed charts' dilated covers are pairwise
              // disjoint (the gutter), and a connected polygon of area A and
              // larger extent E dilated by g covers at least A + 2gE + 4g^2.
              // Once the charts not yet placed cannot fit that way into the
              // area under the frontline, the candidate fails now instead of
              // rows later (checked after every committed row).
              // Charts the prefix-sum tail may draw at its scale count at
              // k - 14 (head_p: those surely drawn at k), and the tail's rows
              // are not checked.
              if (area_bound && row > 0 && !tail) {
                const int hp = ctl.head_p, rs = row_start;
                const unsigned long long p2 = p.pre2[cb + rs], pE = p.preE[cb + rs];
                const unsigned long long h2 = hp < n ? p.pre2[cb + hp] : tot2, hE = hp < n ? p.preE[cb + hp] : totE;
                const int32_t fr = Wp * Hp - ctl.front_sum;  // free texels under the frontline (sides <= 8192)
                const uint64_t kk = 16 * (uint64_t)(j + 1), kr = hybrid ? kk - kTailSteps : kk, gg = (uint64_t)g;
                // at k: the charts from rs to hp; at k - 14: those from max(rs, hp) on
                const unsigned __int128 S2 = rs < hp ? h2 - p2 : 0, SE = rs < hp ? hE - pE : 0;
                const unsigned __int128 R2 = tot2 - (rs < hp ? h2 : p2), RE = totE - (rs < hp ? hE : pE);
                const unsigned __int128 need = S2 * (kk * kk) + R2 * (kr * kr) + (((SE * kk + RE * kr) * (2 * gg)) << 19) +
                                               ((unsigned __int128)(4 * gg * gg * (uint64_t)(n - row_start)) << 37);
                if (need > ((unsigned __int128)(uint32_t)fr << 37)) ctl.bound_fail = 1;
              }
            }
          }
          // per chart: window entries, offsets zeroed
          const int spec = min(n - row_start, maxrow);
          for (int t = tid - 64; t < spec; t += kNT - 64) {
            const int s = row_start + t;
            const int4 mt = *reinterpret_cast<const int4 *>(meta + (int64_t)s * 4);
            wps[t] = mt.x;
            woff[t] = mt.z;
            mbot[t] = mt.w;
            pflw[t] = pfl[s];
            hqw[t] = hqa[s];
#pragma unroll
            for (int cfg = 0; cfg < 8; ++cfg) yb[cfg * maxrow + t] = 0;  // offsets start at 0
          }
        }
        __syncthreads();
        if (ctl.bound_fail) {  // the progressive area bound: the candidate fails
          if (tid == 0) ctl.fail = 1;
          break;
        }
        // The folds examined charts up to the first that does not fit; its
        // position depends on the compaction distance of the pair before it.
        // If that chart is not drawn yet the row waits for the next chunk.
        if (avail < n) {
          const int mx = max(max(ctl.len[0], ctl.len[1]), max(ctl.len[2], ctl.len[3]));
          if (row_start + mx >= avail) {
            deferred = true;
            break;
          }
        }
        if (ctl.len[tail ? vt : 0] == 0) {  // a chart wider than the atlas: this scale fails
          if (tid == 0) ctl.fail = 1;
          break;
        }
        if (tmode == 1) {
          // a tail row folded at the candidate scale: record its charts (the
          // row, and its length at the first) and continue the prefix
          const int len = ctl.len[vt];
          for (int t = tid; t < len; t += kNT)
            place[row_start + t] = make_int4(0, 0, trows, t == 0 ? (len | kTailFirst) : 0);
          if (tid == 0) {
            const int32_t *pos = vt ? posH : posN;
            if (row_start + len < n) {
              ctl.tP = tB + pos[len];
              ctl.tPrev = tB + pos[len - 1];
              ctl.tWprev = wps[len - 1];
              ctl.tHave = 1;
            }
            ctl.trows = trows + 1;
            ctl.row_start = row_start + len;
            ctl.fail = ctl.abort ? 2 : 0;
          }
          __syncthreads();
          continue;
        }

        // ---- D: push ----------------------------------------------------------
        // warp per chart: its TopEdge (and the mirrored one) is loaded once and
        // shared by every configuration the chart takes part in; the per-chart
        // maxima are warp reductions (one instruction per configuration)
        {
          const int len0 = ctl.len[0], len1 = ctl.len[1], len2 = ctl.len[2], len3 = ctl.len[3];
          const int maxlen = max(max(len0, len1), max(len2, len3));
          const int32_t rlo = ctl.region_lo, rhi = ctl.region_hi;
          const int32_t slo = ctl.stage_lo, shi = ctl.stage_hi;
          for (int t = warp; t < maxlen; t += kNW) {
            const int w = wps[t];
            const int32_t cs = woff[t];
            const uint32_t *col = (cs >= slo && cs + w <= shi) ? stage + (cs - slo) : colp + cs;
            const int32_t pn = posN[t], ph = posH[t];
            int32_t X[8];
            X[0] = pn;                X[1] = Wp - pn - w;    // full, side by side
            X[2] = ph;                X[3] = Wp - ph - w;    // full, compacted
            X[4] = rlo + pn;          X[5] = rhi - pn - w;   // knee, side by side
            X[6] = rlo + ph;          X[7] = rhi - ph - w;   // knee, compacted
            const unsigned on = (t < len0 ? 0x03u : 0u) | (t < len1 ? 0x0cu : 0u) |
                                (t < len2 ? 0x30u : 0u) | (t < len3 ? 0xc0u : 0u);
            int32_t acc[8];
#pragma unroll
            for (int cfg = 0; cfg < 8; ++cfg) acc[cfg] = 0;  // offsets start at 0 (the atlas top)
            for (int base = 0; base < w; base += 32) {
              const int i = base + lane;
              if (i < w) {
                const uint32_t f = col[i];
                const uint32_t r = col[w - 1 - i];
                const int32_t tf = (int32_t)(f & 0xffffu), tr = (int32_t)(r & 0xffffu);
#pragma unroll
                for (int cfg = 0; cfg < 4; ++cfg)
                  if ((on >> cfg) & 1u) acc[cfg] = max(acc[cfg], front[X[cfg] + i] - ((cfg & 1) ? tr : tf));
                if (knee) {
#pragma unroll
                  for (int cfg = 4; cfg < 8; ++cfg)
                    if ((on >> cfg) & 1u) acc[cfg] = max(acc[cfg], front[X[cfg] + i] - ((cfg & 1) ? tr : tf));
                }
              }
            }
            int32_t mine = 0;
#pragma unroll
            for (int cfg = 0; cfg < 4; ++cfg) {
              const int32_t m = __reduce_max_sync(0xffffffffu, acc[cfg]);
              if (lane == cfg) mine = m;
            }
            if (knee) {  // the knee configurations exist only while a knee is live
#pragma unroll
              for (int cfg = 4; cfg < 8; ++cfg) {
                const int32_t m = __reduce_max_sync(0xffffffffu, acc[cfg]);
                if (lane == cfg) mine = m;
              }
            }
            if (lane < 8 && ((on >> lane) & 1u)) yb[lane * maxrow + t] = mine;
          }
        }
        __syncthreads();

        // ---- E: interlock fixpoint (Algorithm 2) and scores --------------------
        // warps 0-7: one configuration each; warps 8-9: the knee candidate of the
        // two atlas-width rows (App. A), so selection finds it ready
        if (warp < 8) {
          const int cfg = warp;
          const int v = cfg >> 1, hc = v & 1;
          const int len = ctl.len[v];
          if (len > 0) {
            int32_t *y = yb + cfg * maxrow;
            if (hc) {
              // forward: chart t takes y of t-1 when t cannot move above t-1
              int32_t carry = kI32Min;
              for (int t0 = 0; t0 < len; t0 += 32) {
                const int t = t0 + lane;
                const bool ok = t < len;
                const int32_t yv = ok ? y[t] : kI32Min;
                const bool head = !ok || t == 0 || !(pflw[t - 1] & 2);
                const unsigned heads = __ballot_sync(0xffffffffu, head);
                int32_t f = seg_scan_max(yv, heads | 1u);
                // lanes before the first head of this chunk continue the carry
                const int first_head = heads ? __ffs(heads) - 1 : 32;
                if (lane < first_head) f = max(f, carry);
                carry = __shfl_sync(0xffffffffu, f, 31);
                // forward maxima feed the backward pass: a backward segment's
                // maximum of forward maxima is the maximum over the whole chain
                if (ok) y[t] = f;
                __syncwarp();
              }
              // backward: chart t takes y of t+1 when t cannot move above t+1
              carry = kI32Min;
              const int nchunks = (len + 31) / 32;
              for (int c = nchunks - 1; c >= 0; --c) {
                const int t = c * 32 + (31 - lane);  // reversed lane order
                const bool ok = t < len;
                const int32_t yv = ok ? y[t] : kI32Min;
                const bool head = !ok || t == len - 1 || !(pflw[t] & 1);
                const unsigned heads = __ballot_sync(0xffffffffu, head);
                int32_t b = seg_scan_max(yv, heads | 1u);
                const int first_head = heads ? __ffs(heads) - 1 : 32;
                if (lane < first_head) b = max(b, carry);
                carry = __shfl_sync(0xffffffffu, b, 31);
                __syncwarp();
                if (ok) y[t] = b;
                __syncwarp();
              }
            }
            int32_t mx = kI32Min;
            for (int t = lane; t < len; t += 32) mx = max(mx, y[t] + mbot[t]);
            mx = __reduce_max_sync(0xffffffffu, mx);
            if (lane == 0) {
              ctl.score[cfg] = max(ctl.committed, mx);
              ctl.score_knee[cfg] = knee ? max(ctl.knee_max, mx) : 0;
            }
          }
        } else if (warp < 10 && balance) {
          // largest qualifying unscaled height drop among the first len charts,
          // first on ties (key = drop << 16 | (0xffff - t))
          const int len = ctl.len[warp - 8];
          int64_t key = -1;
          for (int t = lane; t + 1 < len; t += 32) {
            const int64_t D = (int64_t)hqw[t] - hqw[t + 1];
            if (100 * D >= (int64_t)p.knee_abs * 256 * ad.H && 100 * D >= (int64_t)p.knee_rel * hqw[t]) {
              const int64_t kk = (D << 16) | (0xffff - t);
              key = kk > key ? kk : key;
            }
          }
          key = warp_max(key);
          if (lane == 0) ctl.knee_t[warp - 8] = key >= 0 ? 0xffff - (int)(key & 0xffff) : -1;
        }
        __syncthreads();

        // ---- G: selection (Sec. 4.2); the row state advances ------------------
        // Every thread derives the same choice from the scores (fixed since the
        // last barrier) and the row state it read at the row's start; thread 0
        // alone writes the next row's state, which no thread reads before the
        // commit's barrier.
        int best;
        if (tail) {
          best = vt * 2 + (trows % 3 == 0 ? 0 : 1);  // a tail row: FastAtlas's direction pattern
        } else {
          // per fold (0: atlas width, 1: knee): compaction iff it fits more
          // charts, then the direction with the smaller maximum frontline
          int ch[2];
#pragma unroll
          for (int fold = 0; fold < 2; ++fold) {
            const int h = (use_hc && ctl.len[fold * 2 + 1] > ctl.len[fold * 2]) ? 1 : 0;
            const int jl = (fold * 2 + h) * 2, jr = jl + 1;
            const int32_t kl = fold == 0 ? ctl.score[jl] : ctl.score_knee[jl];
            const int32_t kr = fold == 0 ? ctl.score[jr] : ctl.score_knee[jr];
            int dir;
            if (balance) dir = kl < kr ? 0 : (kr < kl ? 1 : (prev_ltr ? 1 : 0));
            else dir = prev_ltr ? 1 : 0;
            ch[fold] = jl + dir;
          }
          best = ch[0];
          if (knee && ctl.len[ch[1] >> 1] > 0 && ctl.score[ch[1]] + p.knee_margin <= ctl.score[best]) best = ch[1];
        }
        if (tid == 0) {
          const int v = best >> 1, dir = best & 1, fold = v >> 1, hc = v & 1;
          const int len = ctl.len[v];
          if (tail) {  // a tail row pushed at the tail scale
            ctl.trows = trows + 1;
          } else if (fold == 0) {
            // App. A: a knee in this row starts the concavity at the taller
            // chart's padded edge; no knee if that concavity would be empty
            int valid = 0;
            const int t = balance ? ctl.knee_t[hc] : -1;
            if (t >= 0) {
              const int32_t X = dir ? Wp - (hc ? posH : posN)[t] - wps[t] : (hc ? posH : posN)[t];
              ctl.knee_ltr = dir == 0;
              ctl.knee_l = X;
              ctl.knee_r = X + wps[t];
              valid = dir == 0 ? (X + wps[t] < Wp) : (X > 0);
            }
            ctl.knee_valid = valid;
            ctl.knees += valid;
          } else {
            ctl.knee_rows += 1;
          }
          ctl.committed = ctl.score[best];
          ctl.fail = ctl.abort ? 2 : (ctl.committed > Hp ? 1 : 0);
          ctl.prev_ltr = dir == 0;
          ctl.row_start = row_start + len;
          ctl.row = row + 1;
        }

        // ---- H: commit ----------------------------------------------------------
        {
          const int v = best >> 1, dir = best & 1, fold = v >> 1, hc = v & 1;
          const int len = ctl.len[v];
          const int32_t lo = fold ? ctl.region_lo : 0, hi = fold ? ctl.region_hi : Wp;
          const int32_t *pos = hc ? posH : posN;
          const int32_t *y = yb + best * maxrow;
          const int32_t slo = ctl.stage_lo, shi = ctl.stage_hi;
          const int fA = woff[0] - slo;
          const int fB = woff[len - 1] + wps[len - 1] - slo;
          int32_t grow = 0;  // this thread's rise of the frontline (telescoping: atomicMax returns the old value)
          if (fB <= shi - slo) {
            for (int f = fA + tid; f < fB; f += kNT) {  // lane per staged column word
              // the word's chart and column, from its staged owner index
              // (checked: a wrong owner raises an error, never a stray access;
              // -1: a word no chart owns, left between the tail's charts when
              // they were redrawn narrower at the tail scale)
              if (sown[f] < 0) continue;
              const int t = sown[f] - row_start;
              if ((unsigned)t >= (unsigned)len) { atomicOr(p.err + at, kErrRow); continue; }
              const int w = wps[t];
              const int i = f - (woff[t] - slo);
              if ((unsigned)i >= (unsigned)w) { atomicOr(p.err + at, kErrRow); continue; }
              const int32_t X = dir ? hi - pos[t] - w : lo + pos[t];
              const int32_t v = y[t] + (int32_t)(stage[f] >> 16);
              if (area_bound) {
                const int32_t old = atomicMax(&front[X + (dir ? w - 1 - i : i)], v);
                grow += v > old ? v - old : 0;
              } else {
                atomicMax(&front[X + (dir ? w - 1 - i : i)], v);
              }
            }
          } else {
          for (int t = warp; t < len; t += kNW) {
            const int w = wps[t];
            const int32_t cs = woff[t];
            const uint32_t *col = (cs >= slo && cs + w <= shi) ? stage + (cs - slo) : colp + cs;
            const int32_t X = dir ? hi - pos[t] - w : lo + pos[t];
            const int32_t yt = y[t];
            for (int i = lane; i < w; i += 32) {
              const uint32_t word = col[dir ? w - 1 - i : i];
              const int32_t v = yt + (int32_t)(word >> 16);
              const int32_t old = atomicMax(&front[X + i], v);
              grow += v > old ? v - old : 0;
            }
          }
          }
          if (area_bound) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) grow += __shfl_xor_sync(0xffffffffu, grow, o);
            if (lane == 0 && grow) atomicAdd(&ctl.front_sum, grow);
          }
          const int bits = dir | (hc << 1) | (fold << 2) | ((int)tail << 3);
          for (int t = tid; t < len; t += kNT) {
            const int32_t X = dir ? hi - pos[t] - wps[t] : lo + pos[t];
            place[row_start + t] = make_int4(X, y[t], row, bits);
          }
          __syncthreads();
        }

      }

      // the tail folded at the candidate scale: park it for the tail search
      const bool parked = !deferred && ctl.tail == 1 && !ctl.fail && ctl.row_start >= n;
      if (deferred || parked) {  // keep the state for the next chunk, or for the tail's push
        for (int x = tid; x < wp_pad; x += kNT) fsave[x] = front[x];
        if (tid == 0) {
          csave[0] = ctl.row_start; csave[1] = ctl.row; csave[2] = ctl.committed; csave[3] = ctl.prev_ltr;
          csave[4] = ctl.knee_valid; csave[5] = ctl.knee_ltr; csave[6] = ctl.knee_l; csave[7] = ctl.knee_r;
          csave[8] = ctl.knee_rows; csave[9] = ctl.knees;
          csave[kCsTail] = ctl.tail | (ctl.tHave << 3) | (ctl.trows << 4);
          csave[11] = ctl.tL; csave[12] = ctl.tP; csave[13] = ctl.tPrev; csave[14] = ctl.tWprev;
          csave[kCsC0] = ctl.c0; csave[kCsHeadRows] = ctl.head_rows; csave[kCsTrows] = ctl.trows;
          csave[kCsCommitted] = ctl.committed;
          p.tstate[at * kScales + j] = parked ? kTaskTailSearch : kTaskRun;
        }
      } else if (tid == 0) {
        const int ok = !ctl.fail && ctl.row_start >= n;
        const bool tailed = ctl.tail == 3;
        so->success = ok;
        so->rows = ctl.row;
        so->knee_rows = ctl.knee_rows;
        so->knees = ctl.knees;
        so->score = ctl.committed;
        so->placed = ctl.row_start;
        so->evaluated = ctl.fail == 2 ? 2 : 1;
        so->tail_rows = ctl.trows;
        so->tail_k = tailed ? ctl.kt : 0;
        so->tail_start = tailed ? ctl.c0 : n;
        if (ok) {
          // Sec. 4.4: the candidate's area-weighted scale sum (its charts at
          // k, the tail's at k'); candidates that cannot exceed it are moot
          const unsigned long long tot = p.area_tot[at];
          const unsigned long long head = tailed ? p.prea[cb + ctl.c0] : tot;
          const unsigned __int128 w = (unsigned __int128)head * (uint64_t)(16 * (j + 1)) +
                                      (unsigned __int128)(tot - head) * (uint64_t)(tailed ? ctl.kt : 0);
          so->wsum[0] = (unsigned long long)w;
          so->wsum[1] = (unsigned long long)(w >> 64);
          atomicMax(p.found + at, moot_below(w, tot));
        }
        p.tstate[at * kScales + j] = kTaskDone;
      }
    }  // task not skipped
    __syncthreads();  // ctl is rewritten by the next task
  }  // task loop
}

}  // namespace

// Shared memory of one row-loop CTA without the column stage.
size_t rowloop_smem_bytes(int W, int g) {
  const int Wp = W + 2 * g;
  const int wp_pad = (Wp + 3) & ~3;
  return sizeof(int32_t) * ((size_t)wp_pad + 15 * (size_t)rowloop_maxrow(W, g)) + sizeof(Ctl) + 64;
}

// ... with a stage of two atlas widths (what an atlas of width W would use).
size_t rowloop_smem_wanted(int W, int g) {
  const int wp_pad = (W + 2 * g + 3) & ~3;
  return rowloop_smem_bytes(W, g) + 2 * sizeof(int32_t) * 2 * (size_t)wp_pad;
}

int rowloop_static_smem() {
  cudaFuncAttributes a;
  int m = 0;
  for (const void *f : {(const void *)rowloop_kernel<1024>, (const void *)rowloop_kernel<512>}) {
    if (cudaFuncGetAttributes(&a, f) != cudaSuccess) return -1;
    m = (int)a.sharedSizeBytes > m ? (int)a.sharedSizeBytes : m;
  }
  return m;
}

cudaError_t rowloop_prepare(int smem) {
  cudaError_t e = cudaFuncSetAttribute(rowloop_kernel<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(rowloop_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

void launch_rowloop(const Pack *dp, const Launch &L, int q, int F, cudaStream_t st) {
  // persistent: as many CTAs as fit on the multiprocessors at once
  if (L.rowloop_threads == 512)
    rowloop_kernel<512><<<L.sms * L.rowloop_ctas, 512, L.rowloop_smem, st>>>(dp, q, F, L.rowloop_smem / 4);
  else
    rowloop_kernel<1024><<<L.sms, 1024, L.rowloop_smem, st>>>(dp, q, F, L.rowloop_smem / 4);
}

}  // namespace tabi
