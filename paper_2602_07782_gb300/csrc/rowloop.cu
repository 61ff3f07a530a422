// Row loop of one candidate scale: Algorithm 5 (with Algorithms 2, 3, 4 and
// the hierarchical selection of Sec. 4.2), one CTA per candidate scale.
//
// Shared memory holds the committed frontline (one int per padded atlas
// column) and the per-row working set.  A row proceeds in barrier-separated
// phases:
//   A  knee refresh (Algorithm 3) and the concavity's current maximum;
//   B  folds (Algorithm 4): warp 0 folds side by side, warp 1 with
//      compaction.  The compacted fold x_{t+1} = max(x_t + w'_t - d_t,
//      x_{t-1} + w'_{t-1}) is a linear recurrence in the (max,+) semiring,
//      evaluated as a warp scan of 2x2 max-plus matrices.  A fold from the
//      same first chart serves both the atlas width and the knee width.
//      Other warps clear the offsets of the previous row;
//   D  push: one warp per chart loads its TopEdge once (both orientations)
//      and forms, for every configuration the chart is part of, the maximum
//      of front[x] - TopEdge over its columns;
//   E  per configuration (one warp each) the interlock fixpoint of
//      Algorithm 2 -- the least solution is, per chart, the maximum pushed
//      offset over the charts chained to it, i.e. a forward and a backward
//      segmented max-scan -- and the score.  After the push the frontline's
//      maximum is max(committed maximum, max_c (y_c + max BottomEdge_c)),
//      so configurations never copy the frontline;
//   G  selection (Sec. 4.2) and knee detection (App. A) by warp 0;
//   H  commit: one warp per chart raises the frontline (shared atomicMax,
//      since compacted neighbours share columns); placements out.
#include "tabi_internal.cuh"

namespace tabi {
namespace {

constexpr int kNT = 512;
constexpr int kNW = kNT / 32;
constexpr int32_t kNeg = -(1 << 28);  // max-plus "minus infinity"
constexpr int32_t kI32Min = -0x7fffffff - 1;

struct Ctl {
  int32_t len[4];        // fold variants v = fold * 2 + hc: charts in the row
  int32_t score[8], score_knee[8];
  int32_t row_start, row, committed, fail, prev_ltr, best, prev_maxlen;
  int32_t knee_valid, knee_ltr, knee_l, knee_r;
  int32_t region_lo, region_hi, knee_max;
  int32_t knee_rows, knees, red[kNW];
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

__device__ __forceinline__ int32_t block_max(int32_t v, Ctl &ctl) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_max(v);
  if (lane == 0) ctl.red[w] = v;
  __syncthreads();
  int32_t r = lane < kNW ? ctl.red[lane] : kI32Min;
  r = warp_max(r);
  __syncthreads();
  return r;
}
__device__ __forceinline__ int32_t block_min(int32_t v, Ctl &ctl) {
  return -block_max(-v, ctl);
}

// segmented inclusive scan (max) over lanes, segments start at head lanes
__device__ __forceinline__ int32_t seg_scan_max(int32_t v, bool head) {
  const int lane = threadIdx.x & 31;
  unsigned hd = head;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t u = __shfl_up_sync(0xffffffffu, v, o);
    const unsigned uh = __shfl_up_sync(0xffffffffu, hd, o);
    if (lane >= o && !hd) v = max(v, u);
    if (lane >= o) hd |= uh;
  }
  return v;
}

__global__ void __launch_bounds__(kNT) rowloop_kernel(Pack p, int j_lo, int maxrow, int wp_pad) {
  const int j = j_lo + blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  ScaleOut *so = p.scale_out + j;
  if (*(volatile int32_t *)p.found >= 0) return;  // a larger scale already succeeded
  if (*(volatile uint32_t *)p.err) return;        // invalid input or pool overflow
  const int n = p.n;
  const int Wp = p.W + 2 * p.g, Hp = p.H + 2 * p.g;
  const uint32_t flags = p.flags;
  const bool use_hc = flags & TABI_F_HC;
  const bool balance = flags & TABI_F_BALANCE;

  extern __shared__ int32_t sm[];
  int32_t *front = sm;                  // [wp_pad]
  int32_t *posN = front + wp_pad;       // [maxrow] side by side
  int32_t *posH = posN + maxrow;        // [maxrow] compacted
  int32_t *yb = posH + maxrow;          // [8][maxrow]
  int32_t *wps = yb + 8 * maxrow;       // [maxrow] w'
  int32_t *mbot = wps + maxrow;         // [maxrow] max BottomEdge
  int32_t *woff = mbot + maxrow;        // [maxrow] pool offset
  __shared__ Ctl ctl;

  const uint32_t *pool = p.pool + (int64_t)j * p.pool_stride;
  const int32_t *meta = p.meta + (int64_t)j * n * 4;
  const int32_t *dnext = p.dnext + (int64_t)j * n;
  const uint8_t *pfl = p.pflags + (int64_t)j * n;
  int4 *place = p.place + (int64_t)j * n;

  for (int x = tid; x < wp_pad; x += kNT) front[x] = 0;
  if (tid == 0) {
    ctl.row_start = 0; ctl.row = 0; ctl.committed = 0; ctl.fail = 0;
    ctl.prev_ltr = 0; ctl.prev_maxlen = 0; ctl.knee_valid = 0;
    ctl.knee_rows = 0; ctl.knees = 0;
  }
  __syncthreads();

  while (true) {
    const int row_start = ctl.row_start;
    if (row_start >= n || ctl.fail) break;

    // ---- A: knee refresh (Algorithm 3) and the concavity's max -----------
    const bool knee = ctl.knee_valid;
    if (knee) {
      const int L = ctl.knee_l, R = ctl.knee_r;
      if (ctl.knee_ltr) {
        const int32_t cur = front[R];
        int32_t best = L - 1;
        for (int x = L + tid; x < R; x += kNT)
          if (front[x] >= cur) best = max(best, x);
        best = block_max(best, ctl);
        if (tid == 0) { ctl.knee_r = best + 1; ctl.region_lo = best + 1; ctl.region_hi = Wp; }
      } else {
        const int32_t cur = front[L - 1];
        int32_t best = R;
        for (int x = L + tid; x < R; x += kNT)
          if (front[x] >= cur) best = min(best, x);
        best = block_min(best, ctl);
        if (tid == 0) { ctl.knee_l = best; ctl.region_lo = 0; ctl.region_hi = best; }
      }
      __syncthreads();
      int32_t mx = 0;
      for (int x = ctl.region_lo + tid; x < ctl.region_hi; x += kNT) mx = max(mx, front[x]);
      mx = block_max(mx, ctl);
      if (tid == 0) ctl.knee_max = mx;
    }

    // ---- B: folds (Algorithm 4) -------------------------------------------
    if (warp < 2) {
      const int hc = warp;  // warp 0: side by side, warp 1: compacted
      const bool active = hc == 0 || use_hc;
      const bool longest = hc == (use_hc ? 1 : 0);
      int32_t lenF = 0, lenK = 0;
      if (active) {
        const int32_t foldF = Wp;
        const int32_t foldK = knee ? ctl.region_hi - ctl.region_lo : -1;
        int32_t *pos = hc ? posH : posN;
        MP carry{0, kNeg, kNeg, 0};  // identity
        int32_t carry_x = 0, carry_wprev = kNeg;
        bool doneF = false, doneK = !knee;
        for (int t0 = 0; !(doneF && doneK); t0 += 32) {
          const int t = t0 + lane;
          const int s = row_start + t;
          const bool valid = s < n;
          const bool room = t < maxrow;  // the last chunk may run past the row capacity
          const int32_t w = valid ? meta[(int64_t)s * 4] : 0;
          int32_t xt, xnext;
          if (hc) {
            const int32_t d = valid ? dnext[s] : 0;
            int32_t wprev = __shfl_up_sync(0xffffffffu, w, 1);
            if (lane == 0) wprev = carry_wprev;
            MP m{w - d, (t == 0) ? kNeg : wprev, 0, kNeg};
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const MP u = mpshfl_up(m, o);
              if (lane >= o) m = mpmul(m, u);
            }
            const MP full = mpmul(m, carry);
            xnext = full.a00;  // applied to the start state (x_0, x_-1) = (0, -inf)
            xt = __shfl_up_sync(0xffffffffu, xnext, 1);
            if (lane == 0) xt = carry_x;
            carry.a00 = __shfl_sync(0xffffffffu, full.a00, 31);
            carry.a01 = __shfl_sync(0xffffffffu, full.a01, 31);
            carry.a10 = __shfl_sync(0xffffffffu, full.a10, 31);
            carry.a11 = __shfl_sync(0xffffffffu, full.a11, 31);
          } else {
            int32_t incl = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const int32_t u = __shfl_up_sync(0xffffffffu, incl, o);
              if (lane >= o) incl += u;
            }
            xnext = carry_x + incl;
            xt = xnext - w;
          }
          // the first chart that does not fit ends the row
          const unsigned overF = __ballot_sync(0xffffffffu, !valid || xt + w > foldF);
          const unsigned overK = __ballot_sync(0xffffffffu, !valid || xt + w > foldK);
          if (!doneF && overF) { lenF = t0 + __ffs(overF) - 1; doneF = true; }
          else if (!doneF) lenF = t0 + 32;
          if (!doneK && overK) { lenK = t0 + __ffs(overK) - 1; doneK = true; }
          else if (!doneK) lenK = t0 + 32;
          if (valid && room) pos[t] = xt;
          if (longest && valid && room) {  // the row window, shared by all configurations
            wps[t] = w;
            mbot[t] = meta[(int64_t)s * 4 + 3];
            woff[t] = meta[(int64_t)s * 4 + 2];
          }
          carry_x = __shfl_sync(0xffffffffu, xnext, 31);
          carry_wprev = __shfl_sync(0xffffffffu, w, 31);
          if (t0 + 32 >= maxrow && !(doneF && doneK)) {  // cannot happen: rows hold <= W'/3 + 1 charts
            if (lane == 0) atomicOr(p.err, kErrRow);
            doneF = doneK = true;
          }
          if ((doneF && lenF >= maxrow) || (doneK && lenK >= maxrow)) {
            if (lane == 0) atomicOr(p.err, kErrRow);
            lenF = min(lenF, maxrow - 1);
            lenK = min(lenK, maxrow - 1);
          }
        }
      }
      if (lane == 0) {
        ctl.len[hc] = active ? lenF : 0;
        ctl.len[2 + hc] = (active && knee) ? lenK : 0;
      }
    }
    __syncthreads();
    if (ctl.len[0] == 0) {  // a chart wider than the atlas: this scale fails
      if (tid == 0) ctl.fail = 1;
      break;
    }

    // ---- D: push ----------------------------------------------------------
    // warp per chart: its TopEdge (and the mirrored one) is loaded once and
    // shared by every configuration the chart takes part in
    {
      const int maxlen = max(max(ctl.len[0], ctl.len[1]), max(ctl.len[2], ctl.len[3]));
      for (int t = warp; t < maxlen; t += kNW) {
        const int w = wps[t];
        const uint32_t *col = pool + woff[t];
        int32_t X[8];
        bool on[8];
#pragma unroll
        for (int cfg = 0; cfg < 8; ++cfg) {
          const int v = cfg >> 1, dir = cfg & 1, fold = v >> 1, hc = v & 1;
          on[cfg] = t < ctl.len[v];
          const int32_t lo = fold ? ctl.region_lo : 0, hi = fold ? ctl.region_hi : Wp;
          const int32_t ps = (hc ? posH : posN)[t];
          X[cfg] = dir ? hi - ps - w : lo + ps;
        }
        int32_t acc[8];
#pragma unroll
        for (int cfg = 0; cfg < 8; ++cfg) acc[cfg] = 0;  // offsets start at 0 (the atlas top)
        for (int base = 0; base < w; base += 32) {
          const int i = base + lane;
          if (i < w) {
            const int32_t tf = (int32_t)(col[i] & 0xffffu);
            const int32_t tr = (int32_t)(col[w - 1 - i] & 0xffffu);
#pragma unroll
            for (int cfg = 0; cfg < 8; ++cfg)
              if (on[cfg]) acc[cfg] = max(acc[cfg], front[X[cfg] + i] - ((cfg & 1) ? tr : tf));
          }
        }
#pragma unroll
        for (int cfg = 0; cfg < 8; ++cfg) {
          const int32_t m = warp_max(acc[cfg]);
          if (on[cfg] && lane == 0) yb[cfg * maxrow + t] = m;
        }
      }
    }
    __syncthreads();

    // ---- E: interlock fixpoint (Algorithm 2) and scores --------------------
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
            const bool head = !ok || t == 0 || !(pfl[row_start + t - 1] & 2);
            int32_t f = seg_scan_max(yv, head || lane == 0);
            // lanes before the first head of this chunk continue the carry
            const unsigned heads = __ballot_sync(0xffffffffu, head);
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
            const bool head = !ok || t == len - 1 || !(pfl[row_start + t] & 1);
            int32_t b = seg_scan_max(yv, head || lane == 0);
            const unsigned heads = __ballot_sync(0xffffffffu, head);
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
        mx = warp_max(mx);
        if (lane == 0) {
          ctl.score[cfg] = max(ctl.committed, mx);
          ctl.score_knee[cfg] = knee ? max(ctl.knee_max, mx) : 0;
        }
      }
    }
    __syncthreads();

    // ---- G: selection (Sec. 4.2) and knee detection (App. A) ---------------
    if (warp == 0) {
      if (lane == 0) {
        int choose[2] = {0, 0};
        const int nfold = knee ? 2 : 1;
        for (int fold = 0; fold < nfold; ++fold) {
          const int h = (use_hc && ctl.len[fold * 2 + 1] > ctl.len[fold * 2]) ? 1 : 0;
          const int jl = (fold * 2 + h) * 2, jr = jl + 1;
          const int32_t kl = fold == 0 ? ctl.score[jl] : ctl.score_knee[jl];
          const int32_t kr = fold == 0 ? ctl.score[jr] : ctl.score_knee[jr];
          int dir;
          if (balance) dir = kl < kr ? 0 : (kr < kl ? 1 : (ctl.prev_ltr ? 1 : 0));
          else dir = ctl.prev_ltr ? 1 : 0;
          choose[fold] = jl + dir;
        }
        int best = choose[0];
        if (knee && ctl.len[choose[1] >> 1] > 0 &&
            ctl.score[choose[1]] + p.knee_margin <= ctl.score[best])
          best = choose[1];
        ctl.best = best;
      }
      __syncwarp();
      const int best = ctl.best;
      const int v = best >> 1, dir = best & 1, fold = v >> 1, hc = v & 1;
      if (fold == 0 && balance) {
        // largest qualifying unscaled height drop in the row, first on ties
        const int len = ctl.len[v];
        int64_t key = -1;
        for (int t = lane; t + 1 < len; t += 32) {
          const int s = row_start + t;
          const int64_t D = (int64_t)p.hq[s] - p.hq[s + 1];
          if (100 * D >= (int64_t)p.knee_abs * 256 * p.H && 100 * D >= (int64_t)p.knee_rel * p.hq[s]) {
            const int64_t kk = (D << 16) | (0xffff - t);
            key = kk > key ? kk : key;
          }
        }
        key = warp_max(key);
        if (lane == 0) {
          int valid = 0;
          if (key >= 0) {
            const int t = 0xffff - (int)(key & 0xffff);
            const int32_t *pos = hc ? posH : posN;
            const int32_t X = dir ? Wp - pos[t] - wps[t] : pos[t];
            ctl.knee_ltr = dir == 0;
            ctl.knee_l = X;
            ctl.knee_r = X + wps[t];
            valid = dir == 0 ? (X + wps[t] < Wp) : (X > 0);
          }
          ctl.knee_valid = valid;
          ctl.knees += valid;
        }
      } else if (fold == 0 && lane == 0) {
        ctl.knee_valid = 0;
      }
    }
    __syncthreads();

    // ---- H: commit ----------------------------------------------------------
    {
      const int best = ctl.best;
      const int v = best >> 1, dir = best & 1, fold = v >> 1, hc = v & 1;
      const int len = ctl.len[v];
      const int32_t lo = fold ? ctl.region_lo : 0, hi = fold ? ctl.region_hi : Wp;
      const int32_t *pos = hc ? posH : posN;
      const int32_t *y = yb + best * maxrow;
      for (int t = warp; t < len; t += kNW) {
        const int w = wps[t];
        const uint32_t *col = pool + woff[t];
        const int32_t X = dir ? hi - pos[t] - w : lo + pos[t];
        const int32_t yt = y[t];
        for (int i = lane; i < w; i += 32) {
          const int32_t bot = (int32_t)(col[dir ? w - 1 - i : i] >> 16);
          atomicMax(&front[X + i], yt + bot);
        }
      }
      const int row = ctl.row;
      const int bits = dir | (hc << 1) | (fold << 2);
      for (int t = tid; t < len; t += kNT) {
        const int32_t X = dir ? hi - pos[t] - wps[t] : lo + pos[t];
        place[row_start + t] = make_int4(X, y[t], row, bits);
      }
      __syncthreads();
      if (tid == 0) {
        const int maxlen = max(max(ctl.len[0], ctl.len[1]), max(ctl.len[2], ctl.len[3]));
        ctl.prev_maxlen = maxlen;
        ctl.committed = ctl.score[best];
        ctl.fail = ctl.committed > Hp;
        ctl.prev_ltr = dir == 0;
        ctl.row_start = row_start + len;
        ctl.row = row + 1;
        if (fold) ctl.knee_rows += 1;
      }
      __syncthreads();
    }
  }

  if (tid == 0) {
    const int ok = !ctl.fail && ctl.row_start >= n;
    so->success = ok;
    so->rows = ctl.row;
    so->knee_rows = ctl.knee_rows;
    so->knees = ctl.knees;
    so->score = ctl.committed;
    so->placed = ctl.row_start;
    so->evaluated = 1;
    if (ok) atomicMax(p.found, j);
  }
}

}  // namespace

// Row capacity: charts in a row start at least 2g + 1 texels apart (each
// padded scanline spans 2g + 1 texels or more), so a row holds at most
// W'/(2g+1) + 1 charts.
static int rowloop_maxrow(int W, int g) {
  const int Wp = W + 2 * g;
  return (Wp / (2 * g + 1) + 2 + 3) & ~3;
}

size_t rowloop_smem_bytes(int W, int g) {
  const int Wp = W + 2 * g;
  const int wp_pad = (Wp + 3) & ~3;
  return sizeof(int32_t) * ((size_t)wp_pad + 13 * (size_t)rowloop_maxrow(W, g)) + sizeof(Ctl);
}

cudaError_t launch_rowloop(const Pack &p, int j_lo, int j_hi, cudaStream_t st) {
  const int Wp = p.W + 2 * p.g;
  const int wp_pad = (Wp + 3) & ~3;
  const int maxrow = rowloop_maxrow(p.W, p.g);
  const size_t smem = sizeof(int32_t) * ((size_t)wp_pad + 13 * (size_t)maxrow);
  cudaError_t e = cudaFuncSetAttribute(rowloop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  rowloop_kernel<<<j_hi - j_lo + 1, kNT, smem, st>>>(p, j_lo, maxrow, wp_pad);
  return cudaGetLastError();
}

}  // namespace tabi
