/*
 * tabi_oracle.c -- plain, slow, sequential CPU oracle for the TABI packing
 * hot path (Gu, Vining, Sheffer, "TABI: Tight and Balanced Interactive Atlas
 * Packing", arXiv 2602.07782).
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA path; the two meet only in the seeded inputs.
 *
 * Every step follows the paper in its own order and is written for a reader
 * to check by eye, with no blocking, fusion or reordering:
 *
 *   prep      Sec. 3.1 + Sec. 4.3: AABB, rotate to taller-than-wide;
 *             Sec. 4.1.1 + App. A "Computing Local AABBs": K slices/axis
 *             (K = 10, App. A; 2 and 5 are the Tab. 13 ablation);
 *             App. A "Computing Chart Orientations": vertical then horizontal
 *             reflection from the slice areas;
 *             Sec. 4.1.1 "merge ... tighter bound": slice refinement;
 *             App. A "Computing Oriented Bounding Boxes": 8 angles in
 *             [0, 7pi/16], minimum-area box.
 *   sort      Sec. 3.1: decreasing AABB height.
 *   envelope  App. A "Parallel Pushing Algorithm": TopEdge/BottomEdge per
 *             texel column as the tighter of the two proxies, top rounded
 *             outward, bottom rounded outward; the same per texel row
 *             (left/right extents) for horizontal compaction; Sec. 5 gutters.
 *   hcompact  Sec. 4.1.2 compacting distance; App. A "Detecting Interlocking
 *             Charts" (CannotMoveAbove).
 *   row loop  Algorithm 5 with Algorithm 4 (FoldRow), Algorithm 2
 *             (CorrectYOffsets, the literal do-while), Algorithm 3
 *             (UpdateKneeLocation), knee detection (App. A "Knee Detection
 *             Parameters") and the hierarchical selection of Sec. 4.2.
 *   hybrid    Sec. 4.4: past the rows with knees and tall charts, the rest
 *             of the charts are folded by a prefix sum of their offsets and
 *             pushed row by row in a fixed direction pattern.
 *   search    Sec. 3.1 / Sec. 5: 64 candidate scales, largest success wins.
 *
 * Integer conventions (the paper fixes no precision):
 *   vertices are int32 in 1/256 texel ("Q.8"); a candidate scale is k/1024
 *   with k = 16j, j = 1..64 (the paper's 1/64..64/64); a scaled coordinate is
 *   Q.8 * k, i.e. units of 2^-18 texel, exact in 64 bits.  y grows downward,
 *   0 is the atlas top (Algorithm 2 comment).  Every step is integer.
 *
 * Where the paper is silent or ambiguous, the reading taken here is marked
 * "READING:" and is the same reading the CUDA path implements.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_K 10          /* most local AABBs per axis (App. A default; Tab. 13
                            ablates 2 and 5); the count K is a parameter    */
#define OR_ANGLES 8      /* OBB rotations m*pi/16, m = 0..7 (App. A)          */
#define OR_REC 128       /* int64 fields per chart record                    */
#define OR_FIX 262144LL  /* 2^18: scaled units per texel                     */

typedef __int128 i128;

/* ---- chart record layout (int64 fields), shared with the Python wrapper -- */
enum {
  R_ORIG = 0, R_MINX, R_MINY, R_W0, R_H0, R_WQ, R_HQ, R_ROT, R_FLIPY, R_FLIPX,
  R_OBBM = 10, R_U0, R_U1, R_V0, R_V1,
  R_X = 15,            /* X[0..K]   x-slice boundaries          */
  R_Y = 26,            /* Y[0..K]   y-slice boundaries          */
  R_YLO = 37, R_YHI = 47, R_XLO = 57, R_XHI = 67,  /* raw final slices      */
  R_TLO = 77, R_BHI = 87, R_LLO = 97, R_RHI = 107, /* refined pieces        */
  R_ATOP = 117, R_ABOT, R_ALEFT, R_ARIGHT, R_ABL2, R_ABR2,
  R_LK = 123           /* K: local AABBs per axis of this record         */
};

/* ---- params (int32 array) ------------------------------------------------ */
enum { P_GUTTER = 0, P_KNEE_ABS, P_KNEE_REL, P_LR_SIG, P_KNEE_MARGIN, P_FLAGS, P_LAABB_K,
       P_TOPT, P_HYBRID_MIN, P_COUNT };
#define F_HC      1  /* horizontal compacting configurations (Sec. 4.1.2)       */
#define F_BALANCE 2  /* direction choice + knees (Sec. 4.2); else alternation   */
#define F_OBB     4  /* OBB proxy in the envelope (Sec. 4.1.1)                  */
#define F_LAABB   8  /* local-AABB proxy in the envelope; both off = boxes only */

/* ------------------------------------------------------------------------ */
/* exact rational rounding                                                  */
/* ------------------------------------------------------------------------ */
static int64_t floor_div(i128 a, i128 b) {        /* b > 0 */
  i128 q = a / b;
  if ((a % b) != 0 && a < 0) q -= 1;
  return (int64_t)q;
}
static int64_t ceil_div(i128 a, i128 b) {         /* b > 0 */
  i128 q = a / b;
  if ((a % b) != 0 && a > 0) q += 1;
  return (int64_t)q;
}
static int64_t mn64(int64_t a, int64_t b) { return a < b ? a : b; }
static int64_t mx64(int64_t a, int64_t b) { return a > b ? a : b; }

/* ------------------------------------------------------------------------ */
/* Sec. 4.1.1 local AABB of one slice: floor(min v) and ceil(max v) over the */
/* points of the polygon whose u lies in the closed slab [a, b].  The extreme */
/* values of a closed polygon over a slab are reached on its boundary, and on */
/* one edge at a clipped end point, so every edge is clipped to the slab and */
/* its two end values (exact rationals) are rounded outward.                 */
/* ------------------------------------------------------------------------ */
static int slab_extent(int nv, const int64_t *u, const int64_t *v,
                       int64_t a, int64_t b, int64_t *lo, int64_t *hi) {
  int found = 0;
  int64_t mn = INT64_MAX, mx = INT64_MIN;
  for (int e = 0; e < nv; ++e) {
    int64_t u0 = u[e], v0 = v[e];
    int64_t u1 = u[(e + 1) % nv], v1 = v[(e + 1) % nv];
    if (u0 == u1) {
      if (u0 >= a && u0 <= b) {
        mn = mn64(mn, mn64(v0, v1));
        mx = mx64(mx, mx64(v0, v1));
        found = 1;
      }
      continue;
    }
    int64_t ul = mn64(u0, u1), ur = mx64(u0, u1);
    int64_t ca = mx64(a, ul), cb = mn64(b, ur);
    if (ca > cb) continue;
    int64_t ends[2] = {ca, cb};
    for (int t = 0; t < 2; ++t) {
      /* v at u = ends[t] on the line through (u0,v0),(u1,v1) */
      i128 num = (i128)v0 * (u1 - u0) + (i128)(ends[t] - u0) * (v1 - v0);
      i128 den = (i128)(u1 - u0);
      if (den < 0) { num = -num; den = -den; }
      mn = mn64(mn, floor_div(num, den));
      mx = mx64(mx, ceil_div(num, den));
    }
    found = 1;
  }
  *lo = mn;
  *hi = mx;
  return found;
}

/* K equal intervals per axis: boundaries floor(i*extent/K); slice i is the  */
/* closed interval [X_i, X_{i+1}].  READING: equal widths up to flooring.    */
static int local_aabbs(int K, int nv, const int64_t *x, const int64_t *y, int64_t Wq, int64_t Hq,
                       int64_t *X, int64_t *Y, int64_t *ylo, int64_t *yhi,
                       int64_t *xlo, int64_t *xhi) {
  for (int i = 0; i <= K; ++i) {
    X[i] = (int64_t)i * Wq / K;
    Y[i] = (int64_t)i * Hq / K;
  }
  int ok = 1;
  for (int i = 0; i < K; ++i)
    ok &= slab_extent(nv, x, y, X[i], X[i + 1], &ylo[i], &yhi[i]);
  for (int j = 0; j < K; ++j)
    ok &= slab_extent(nv, y, x, Y[j], Y[j + 1], &xlo[j], &xhi[j]);
  return ok;
}

/* OBB angle table: C_m, S_m = round-half-away(2^14 cos/sin(m*pi/16)).        */
static void obb_table(int64_t *C, int64_t *S) {
  const double pi = 3.14159265358979323846;
  for (int m = 0; m < OR_ANGLES; ++m) {
    C[m] = llround(16384.0 * cos(m * pi / 16.0));
    S[m] = llround(16384.0 * sin(m * pi / 16.0));
  }
}

void oracle_obb_table(int64_t *out /* 16 */) {
  obb_table(out, out + OR_ANGLES);
}

/* ------------------------------------------------------------------------ */
/* prep of one chart (input order)                                          */
/* ------------------------------------------------------------------------ */
static int prep_one(int nv, const int32_t *v, const int32_t *params, int64_t *r) {
  memset(r, 0, sizeof(int64_t) * OR_REC);
  const int K = params[P_LAABB_K];
  if (nv < 3 || K < 1 || K > OR_K) return 1;
  r[R_LK] = K;
  int64_t *x = (int64_t *)malloc(sizeof(int64_t) * nv);
  int64_t *y = (int64_t *)malloc(sizeof(int64_t) * nv);

  /* Sec. 3.1: the chart's AABB */
  int64_t minx = v[0], maxx = v[0], miny = v[1], maxy = v[1];
  for (int i = 1; i < nv; ++i) {
    minx = mn64(minx, v[2 * i]); maxx = mx64(maxx, v[2 * i]);
    miny = mn64(miny, v[2 * i + 1]); maxy = mx64(maxy, v[2 * i + 1]);
  }
  int64_t W0 = maxx - minx, H0 = maxy - miny;
  r[R_MINX] = minx; r[R_MINY] = miny; r[R_W0] = W0; r[R_H0] = H0;

  /* Sec. 3.1: rotate by 90 degrees if wider than tall (READING: strictly),  */
  /* mapping the translated point (x, y) to (y, W0 - x).                      */
  int rot = W0 > H0;
  for (int i = 0; i < nv; ++i) {
    int64_t tx = v[2 * i] - minx, ty = v[2 * i + 1] - miny;
    if (rot) { x[i] = ty; y[i] = W0 - tx; }
    else     { x[i] = tx; y[i] = ty; }
  }
  int64_t Wq = rot ? H0 : W0, Hq = rot ? W0 : H0;
  r[R_ROT] = rot; r[R_WQ] = Wq; r[R_HQ] = Hq;
  if (Wq < 256 || Hq < 256) { free(x); free(y); return 1; }

  int64_t X[OR_K + 1], Y[OR_K + 1], ylo[OR_K], yhi[OR_K], xlo[OR_K], xhi[OR_K];

  /* App. A "Computing Chart Orientations": top and bottom empty areas between */
  /* the x-slices' bounds and the AABB; reflect vertically if top > bottom.    */
  local_aabbs(K, nv, x, y, Wq, Hq, X, Y, ylo, yhi, xlo, xhi);
  int64_t top = 0, bottom = 0;
  for (int i = 0; i < K; ++i) {
    top += (X[i + 1] - X[i]) * ylo[i];
    bottom += (X[i + 1] - X[i]) * (Hq - yhi[i]);
  }
  int flip_y = top > bottom;
  if (flip_y)
    for (int i = 0; i < nv; ++i) y[i] = Hq - y[i];
  r[R_ATOP] = top; r[R_ABOT] = bottom; r[R_FLIPY] = flip_y;

  /* Then left/right areas from the y-slices (READING: recomputed on the     */
  /* vertically reflected chart).  Reflect horizontally if left exceeds right */
  /* by more than lr_sig percent of the AABB area; if neither side is         */
  /* significantly larger, reflect when the bottom area left of the midline  */
  /* exceeds the bottom area right of it (READING: strict; the midline split */
  /* is exact in doubled coordinates).                                        */
  local_aabbs(K, nv, x, y, Wq, Hq, X, Y, ylo, yhi, xlo, xhi);
  int64_t left = 0, right = 0, bl2 = 0, br2 = 0;
  for (int j = 0; j < K; ++j) {
    left += (Y[j + 1] - Y[j]) * xlo[j];
    right += (Y[j + 1] - Y[j]) * (Wq - xhi[j]);
  }
  for (int i = 0; i < K; ++i) {
    int64_t e = Hq - yhi[i];
    int64_t a2 = 2 * X[i], b2 = 2 * X[i + 1];
    int64_t lenL = mx64(0, mn64(b2, Wq) - mx64(a2, 0));
    int64_t lenR = mx64(0, mn64(b2, 2 * Wq) - mx64(a2, Wq));
    bl2 += e * lenL;
    br2 += e * lenR;
  }
  int64_t diff = left - right;
  int64_t adiff = diff < 0 ? -diff : diff;
  int flip_x;
  if ((i128)100 * adiff > (i128)params[P_LR_SIG] * Wq * Hq) flip_x = diff > 0;
  else flip_x = bl2 > br2;
  if (flip_x)
    for (int i = 0; i < nv; ++i) x[i] = Wq - x[i];
  r[R_ALEFT] = left; r[R_ARIGHT] = right; r[R_ABL2] = bl2; r[R_ABR2] = br2;
  r[R_FLIPX] = flip_x;

  /* final local AABBs on the reflected chart */
  local_aabbs(K, nv, x, y, Wq, Hq, X, Y, ylo, yhi, xlo, xhi);
  for (int i = 0; i <= K; ++i) { r[R_X + i] = X[i]; r[R_Y + i] = Y[i]; }
  for (int i = 0; i < K; ++i) {
    r[R_YLO + i] = ylo[i]; r[R_YHI + i] = yhi[i];
    r[R_XLO + i] = xlo[i]; r[R_XHI + i] = xhi[i];
  }

  /* Sec. 4.1.1 merge: each x-slice's top (bottom) is tightened by the first */
  /* (last) y-slice whose x-range meets it; each y-slice's left (right) by   */
  /* the first (last) x-slice whose y-range meets it.  READING: the merge is */
  /* a per-slice refinement, closed-interval intersection tests.             */
  for (int i = 0; i < K; ++i) {
    int64_t t2 = INT64_MAX, b2v = INT64_MIN;
    for (int j = 0; j < K; ++j)
      if (xlo[j] <= X[i + 1] && xhi[j] >= X[i]) {
        t2 = mn64(t2, Y[j]);
        b2v = mx64(b2v, Y[j + 1]);
      }
    r[R_TLO + i] = mx64(ylo[i], t2);
    r[R_BHI + i] = mn64(yhi[i], b2v);
  }
  for (int j = 0; j < K; ++j) {
    int64_t l2 = INT64_MAX, r2 = INT64_MIN;
    for (int i = 0; i < K; ++i)
      if (ylo[i] <= Y[j + 1] && yhi[i] >= Y[j]) {
        l2 = mn64(l2, X[i]);
        r2 = mx64(r2, X[i + 1]);
      }
    r[R_LLO + j] = mx64(xlo[j], l2);
    r[R_RHI + j] = mn64(xhi[j], r2);
  }

  /* App. A "Computing Oriented Bounding Boxes": for each of 8 angles the    */
  /* box is the intersection of the strips u in [u0,u1], v in [v0,v1] with   */
  /* u = xC + yS, v = -xS + yC over the vertices; keep the minimum area      */
  /* (u1-u0)(v1-v0)/(C^2+S^2), compared exactly; ties keep the smaller m.    */
  int64_t C[OR_ANGLES], S[OR_ANGLES];
  obb_table(C, S);
  int best = -1;
  i128 best_area = 0, best_n = 1;
  int64_t bu0 = 0, bu1 = 0, bv0 = 0, bv1 = 0;
  for (int m = 0; m < OR_ANGLES; ++m) {
    int64_t u0 = INT64_MAX, u1 = INT64_MIN, v0 = INT64_MAX, v1 = INT64_MIN;
    for (int i = 0; i < nv; ++i) {
      int64_t uu = x[i] * C[m] + y[i] * S[m];
      int64_t vv = -x[i] * S[m] + y[i] * C[m];
      u0 = mn64(u0, uu); u1 = mx64(u1, uu);
      v0 = mn64(v0, vv); v1 = mx64(v1, vv);
    }
    i128 area = (i128)(u1 - u0) * (v1 - v0);
    i128 nrm = (i128)C[m] * C[m] + (i128)S[m] * S[m];
    if (best < 0 || area * best_n < best_area * nrm) {
      best = m; best_area = area; best_n = nrm;
      bu0 = u0; bu1 = u1; bv0 = v0; bv1 = v1;
    }
  }
  r[R_OBBM] = best; r[R_U0] = bu0; r[R_U1] = bu1; r[R_V0] = bv0; r[R_V1] = bv1;
  free(x);
  free(y);
  return 0;
}

/* Input validation shared by the oracle entry points: returns 0 if valid. */
static int validate(int32_t n, const uint32_t *offsets, const int32_t *verts) {
  if (n < 1) return 1;
  for (int c = 0; c < n; ++c) {
    if (offsets[c + 1] < offsets[c] || offsets[c + 1] - offsets[c] < 3) return 1;
    for (uint32_t i = offsets[c]; i < offsets[c + 1]; ++i) {
      int32_t vx = verts[2 * i], vy = verts[2 * i + 1];
      if (vx <= -(1 << 20) || vx >= (1 << 20) || vy <= -(1 << 20) || vy >= (1 << 20)) return 1;
    }
  }
  return 0;
}

int oracle_prep(int32_t n, const uint32_t *offsets, const int32_t *verts,
                const int32_t *params, int64_t *rec) {
  if (validate(n, offsets, verts)) return 1;
  for (int c = 0; c < n; ++c) {
    int nv = (int)(offsets[c + 1] - offsets[c]);
    if (prep_one(nv, verts + 2 * offsets[c], params, rec + (int64_t)c * OR_REC)) return 1;
    rec[(int64_t)c * OR_REC + R_ORIG] = c;
  }
  return 0;
}

/* Sec. 3.1: sort by AABB height, decreasing.  READING: ties keep the input */
/* order (insertion sort: plainly stable).                                  */
void oracle_sort(int32_t n, const int64_t *rec, int32_t *perm) {
  for (int i = 0; i < n; ++i) perm[i] = i;
  for (int i = 1; i < n; ++i) {
    int32_t p = perm[i];
    int64_t h = rec[(int64_t)p * OR_REC + R_HQ];
    int j = i - 1;
    while (j >= 0 && rec[(int64_t)perm[j] * OR_REC + R_HQ] < h) {
      perm[j + 1] = perm[j];
      --j;
    }
    perm[j + 1] = p;
  }
}

/* ------------------------------------------------------------------------ */
/* envelopes at scale k                                                      */
/* ------------------------------------------------------------------------ */
/* Scaled chart size in texels: w = ceil(Wq*k/2^18), h likewise.             */
static int64_t scaled_len(int64_t q, int64_t k) { return ceil_div((i128)q * k, OR_FIX); }

/* READING of App. A "TopEdge ... BottomEdge": over texel column c (the open  */
/* interval (c, c+1), clipped to the chart's x-range) TopEdge is the floor of */
/* the least y of the tighter proxy and BottomEdge the ceiling of the        */
/* greatest y ("rounded" outward so separation stays strict).  The local-    */
/* AABB proxy contributes the refined pieces whose open x-interval meets the */
/* column; the OBB contributes the minimum (maximum) of its top (bottom)     */
/* boundary over the column, reached at the box corner when the corner lies  */
/* inside the column and at the nearer column end otherwise (each boundary   */
/* is the max (min) of two lines).  The per-row left/right extents are the   */
/* same construction with the axes swapped.                                  */
int oracle_envelope(const int64_t *r, int32_t k, const int32_t *params, int32_t *wh,
                    int32_t *top, int32_t *bot, int32_t *left, int32_t *right, int32_t cap) {
  const int64_t F = OR_FIX;
  int64_t Wq = r[R_WQ], Hq = r[R_HQ];
  int64_t w = scaled_len(Wq, k), h = scaled_len(Hq, k);
  wh[0] = (int32_t)w;
  wh[1] = (int32_t)h;
  if (w > cap || h > cap) return 1;
  int flags = params[P_FLAGS];
  int use_l = (flags & F_LAABB) != 0, use_o = (flags & F_OBB) != 0;
  const int K = (int)r[R_LK];
  int64_t C[OR_ANGLES], S[OR_ANGLES];
  obb_table(C, S);
  int m = (int)r[R_OBBM];
  i128 Cm = C[m], Sm = S[m], N = Cm * Cm + Sm * Sm;
  i128 U0 = (i128)r[R_U0] * k, U1 = (i128)r[R_U1] * k;
  i128 V0 = (i128)r[R_V0] * k, V1 = (i128)r[R_V1] * k;

  for (int64_t c = 0; c < w; ++c) {
    int64_t a = c * F, b = mn64((c + 1) * F, Wq * k);
    int64_t T = 0, B = h;
    if (use_l) {
      int64_t tl = INT64_MAX, bl = INT64_MIN;
      for (int i = 0; i < K; ++i)
        if (r[R_X + i] * k < b && r[R_X + i + 1] * k > a) {
          tl = mn64(tl, r[R_TLO + i]);
          bl = mx64(bl, r[R_BHI + i]);
        }
      T = mx64(T, floor_div((i128)tl * k, F));
      B = mn64(B, ceil_div((i128)bl * k, F));
    }
    if (use_o && m > 0) {
      /* top boundary y(X) = max((U0 - X C)/S, (V0 + X S)/C), corner u=U0, v=V0 */
      i128 xc = U0 * Cm - V0 * Sm; /* corner X times N */
      int64_t to;
      if ((i128)a * N <= xc && xc <= (i128)b * N) {
        to = floor_div(U0 * Sm + V0 * Cm, N * F);
      } else {
        int64_t Xe = (xc < (i128)a * N) ? a : b;
        to = mx64(floor_div(U0 - (i128)Xe * Cm, Sm * F), floor_div(V0 + (i128)Xe * Sm, Cm * F));
      }
      /* bottom boundary y(X) = min((U1 - X C)/S, (V1 + X S)/C), corner u=U1, v=V1 */
      i128 xb = U1 * Cm - V1 * Sm;
      int64_t bo;
      if ((i128)a * N <= xb && xb <= (i128)b * N) {
        bo = ceil_div(U1 * Sm + V1 * Cm, N * F);
      } else {
        int64_t Xe = (xb < (i128)a * N) ? a : b;
        bo = mn64(ceil_div(U1 - (i128)Xe * Cm, Sm * F), ceil_div(V1 + (i128)Xe * Sm, Cm * F));
      }
      T = mx64(T, to);
      B = mn64(B, bo);
    }
    /* READING: keep each column a non-empty interval inside [0, h] */
    T = mx64(0, mn64(T, h - 1));
    B = mx64(T + 1, mn64(B, h));
    top[c] = (int32_t)T;
    bot[c] = (int32_t)B;
  }

  for (int64_t rr = 0; rr < h; ++rr) {
    int64_t a = rr * F, b = mn64((rr + 1) * F, Hq * k);
    int64_t L = 0, R = w;
    if (use_l) {
      int64_t ll = INT64_MAX, rl = INT64_MIN;
      for (int j = 0; j < K; ++j)
        if (r[R_Y + j] * k < b && r[R_Y + j + 1] * k > a) {
          ll = mn64(ll, r[R_LLO + j]);
          rl = mx64(rl, r[R_RHI + j]);
        }
      L = mx64(L, floor_div((i128)ll * k, F));
      R = mn64(R, ceil_div((i128)rl * k, F));
    }
    if (use_o && m > 0) {
      /* left boundary x(Y) = max((U0 - Y S)/C, (Y C - V1)/S), corner u=U0, v=V1 */
      i128 yc = U0 * Sm + V1 * Cm;
      int64_t lo;
      if ((i128)a * N <= yc && yc <= (i128)b * N) {
        lo = floor_div(U0 * Cm - V1 * Sm, N * F);
      } else {
        int64_t Ye = (yc < (i128)a * N) ? a : b;
        lo = mx64(floor_div(U0 - (i128)Ye * Sm, Cm * F), floor_div((i128)Ye * Cm - V1, Sm * F));
      }
      /* right boundary x(Y) = min((U1 - Y S)/C, (Y C - V0)/S), corner u=U1, v=V0 */
      i128 yr = U1 * Sm + V0 * Cm;
      int64_t ro;
      if ((i128)a * N <= yr && yr <= (i128)b * N) {
        ro = ceil_div(U1 * Cm - V0 * Sm, N * F);
      } else {
        int64_t Ye = (yr < (i128)a * N) ? a : b;
        ro = mn64(ceil_div(U1 - (i128)Ye * Sm, Cm * F), ceil_div((i128)Ye * Cm - V0, Sm * F));
      }
      L = mx64(L, lo);
      R = mn64(R, ro);
    }
    L = mx64(0, mn64(L, w - 1));
    R = mx64(L + 1, mn64(R, w));
    left[rr] = (int32_t)L;
    right[rr] = (int32_t)R;
  }
  return 0;
}

/* Sec. 5 gutters (g texels around each chart, none at the atlas edges).     */
/* READING: each envelope is dilated by g in the Chebyshev sense into padded */
/* coordinates (width w+2g, height h+2g); padded footprints must be disjoint */
/* inside the padded atlas (W+2g) x (H+2g).  A chart whose padded footprint  */
/* starts at padded (X, Y) has its texels at atlas (X, Y) onward.            */
int oracle_envelope_padded(const int64_t *r, int32_t k, const int32_t *params, int32_t *wh,
                           int32_t *topP, int32_t *botP, int32_t *leftP, int32_t *rightP,
                           int32_t cap) {
  int g = params[P_GUTTER];
  int64_t w = scaled_len(r[R_WQ], k), h = scaled_len(r[R_HQ], k);
  if (w > cap || h > cap) { wh[0] = (int32_t)w; wh[1] = (int32_t)h; return 1; }
  int32_t *t = (int32_t *)malloc(sizeof(int32_t) * (w + h + 2));
  int32_t *bo = (int32_t *)malloc(sizeof(int32_t) * (w + 1));
  int32_t *l = (int32_t *)malloc(sizeof(int32_t) * (h + 1));
  int32_t *ri = (int32_t *)malloc(sizeof(int32_t) * (h + 1));
  int32_t whr[2];
  oracle_envelope(r, k, params, whr, t, bo, l, ri, cap);
  int64_t wp = w + 2 * g, hp = h + 2 * g;
  wh[0] = (int32_t)wp;
  wh[1] = (int32_t)hp;
  if (wp > cap || hp > cap) { free(t); free(bo); free(l); free(ri); return 1; }
  for (int64_t i = 0; i < wp; ++i) {
    int64_t mnv = INT64_MAX, mxv = INT64_MIN;
    for (int64_t c = i - 2 * g; c <= i; ++c)
      if (c >= 0 && c < w) { mnv = mn64(mnv, t[c]); mxv = mx64(mxv, bo[c]); }
    topP[i] = (int32_t)mnv;
    botP[i] = (int32_t)(mxv + 2 * g);
  }
  for (int64_t i = 0; i < hp; ++i) {
    int64_t mnv = INT64_MAX, mxv = INT64_MIN;
    for (int64_t rr = i - 2 * g; rr <= i; ++rr)
      if (rr >= 0 && rr < h) { mnv = mn64(mnv, l[rr]); mxv = mx64(mxv, ri[rr]); }
    leftP[i] = (int32_t)mnv;
    rightP[i] = (int32_t)(mxv + 2 * g);
  }
  free(t); free(bo); free(l); free(ri);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.1.2 compacting distance and App. A interlock flags for the pair   */
/* (A, B) lined up top-aligned, B right of A.  READING: distances come from */
/* the per-row left/right extents of the combined (tighter) proxy, which is */
/* at least as large as either proxy's own distance and still safe.        */
/*   d = max shift of B toward A: w'_A - max_r (R'_A(r) - L'_B(r))           */
/*   B may move up relative to A iff, for every row r of B, B's left edge   */
/*     stays right of every row of A above r;                               */
/*   A may move up relative to B iff, for every row r of A, A's right edge  */
/*     stays left of every row of B above r.                                */
/* out[0] = d, out[1] = CannotMoveAbove(A, B), out[2] = CannotMoveAbove(B, A) */
/* ------------------------------------------------------------------------ */
static void hcompact_env(int32_t wA, int32_t hA, const int32_t *RA,
                         int32_t hB, const int32_t *LB, int32_t *out) {
  int32_t hmin = hA < hB ? hA : hB;
  int64_t M = INT64_MIN;
  for (int r = 0; r < hmin; ++r) M = mx64(M, (int64_t)RA[r] - LB[r]);
  int64_t d = (int64_t)wA - M;
  if (d < 0) d = 0;
  int64_t off = (int64_t)wA - d; /* B's padded origin relative to A's */
  int b_free = 1;
  int64_t pm = INT64_MIN; /* max of R'_A over the rows of A above row r */
  for (int r = 0; r < hB; ++r) {
    if (r > 0 && off + LB[r] < pm) b_free = 0;
    if (r < hA) pm = mx64(pm, RA[r]);
  }
  int a_free = 1;
  int64_t pmin = INT64_MAX; /* min of B's left edge over the rows of B above row r */
  for (int r = 0; r < hA; ++r) {
    if (r > 0 && RA[r] > pmin) a_free = 0;
    if (r < hB) pmin = mn64(pmin, off + LB[r]);
  }
  out[0] = (int32_t)d;
  out[1] = !a_free;
  out[2] = !b_free;
}

int oracle_hcompact(const int64_t *ra, const int64_t *rb, int32_t k, const int32_t *params,
                    int32_t *out) {
  int32_t cap = 1 << 15;
  int32_t *bufA = (int32_t *)malloc(sizeof(int32_t) * 4 * cap);
  int32_t *bufB = (int32_t *)malloc(sizeof(int32_t) * 4 * cap);
  int32_t whA[2], whB[2];
  int e = oracle_envelope_padded(ra, k, params, whA, bufA, bufA + cap, bufA + 2 * cap, bufA + 3 * cap, cap);
  e |= oracle_envelope_padded(rb, k, params, whB, bufB, bufB + cap, bufB + 2 * cap, bufB + 3 * cap, cap);
  if (!e) hcompact_env(whA[0], whA[1], bufA + 3 * cap, whB[1], bufB + 2 * cap, out);
  free(bufA);
  free(bufB);
  return e;
}

/* ------------------------------------------------------------------------ */
/* one candidate scale: Algorithm 5                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t wp, hp;         /* padded size */
  int32_t *top, *bot;     /* padded column envelope, wp entries */
  int32_t *left, *right;  /* padded row envelope, hp entries    */
} Env;

typedef struct { int valid, ltr; int32_t left, right; } Knee;

/* Algorithm 4 FoldRow.  Returns the last chart index in the row (rowStart-1 */
/* for an empty row) and each chart's left edge relative to the row start.   */
/* READING (added): with compacting on, a chart never starts left of the    */
/* right edge of the chart two places before it, so only neighbours share   */
/* columns and the pairwise interlock of Algorithm 2 is enough to keep the  */
/* row overlap-free.                                                        */
static int fold_row(int n, int s0, int64_t foldW, int hc, const Env *env,
                    const int32_t *dnext, int64_t *pos) {
  int64_t x = 0;
  int64_t prev_right = INT64_MIN;
  for (int s = s0; s < n; ++s) {
    int64_t next_left = x + env[s].wp;
    if (next_left > foldW) return s - 1;
    pos[s] = x;
    if (hc) {
      int64_t nx = next_left - dnext[s];
      if (nx < prev_right) nx = prev_right;
      prev_right = next_left;
      x = nx;
    } else {
      x = next_left;
    }
  }
  return n - 1;
}

/* Algorithm 2 CorrectYOffsets, the literal do-while. */
static void correct_y_offsets(int s0, int s1, const uint8_t *cannotA, const uint8_t *cannotB,
                              int64_t *y) {
  int violation;
  do {
    violation = 0;
    for (int s = s0; s < s1; ++s) {
      if (cannotA[s] && y[s] < y[s + 1]) { violation = 1; y[s] = mx64(y[s], y[s + 1]); }
      if (cannotB[s] && y[s + 1] < y[s]) { violation = 1; y[s + 1] = mx64(y[s + 1], y[s]); }
    }
  } while (violation);
}

/* Algorithm 3 UpdateKneeLocation. */
static void update_knee(Knee *kd, const int64_t *front) {
  if (kd->ltr) {
    int64_t cur = front[kd->right];
    int64_t nk = kd->left - 1;
    for (int64_t x = kd->left; x < kd->right; ++x)
      if (front[x] >= cur) nk = mx64(nk, x);
    kd->right = (int32_t)(nk + 1);
  } else {
    int64_t cur = front[kd->left - 1];
    int64_t nk = kd->right;
    for (int64_t x = kd->left; x < kd->right; ++x)
      if (front[x] >= cur) nk = mn64(nk, x);
    kd->left = (int32_t)nk;
  }
}

/* App. A "Knee Detection Parameters": consecutive charts of the committed  */
/* row whose unscaled height drop is at least knee_abs% of the atlas height */
/* and knee_rel% of the taller chart; the largest drop wins (READING: ties  */
/* keep the first).  The taller chart's concavity-facing edge starts the    */
/* concavity (right edge for a left-to-right row, left edge otherwise).     */
static Knee find_knee(int s0, int s1, int ltr, const int64_t *X, const Env *env,
                      const int64_t *hq, int32_t atlasH, int32_t Wp, const int32_t *params) {
  Knee kd = {0, ltr, 0, 0};
  int best = -1;
  int64_t bestD = 0;
  for (int s = s0; s < s1; ++s) {
    int64_t D = hq[s] - hq[s + 1];
    if (100 * D >= (int64_t)params[P_KNEE_ABS] * 256 * atlasH &&
        100 * D >= (int64_t)params[P_KNEE_REL] * hq[s] && D > bestD) {
      best = s;
      bestD = D;
    }
  }
  if (best < 0) return kd;
  kd.left = (int32_t)X[best];
  kd.right = (int32_t)(X[best] + env[best].wp);
  /* READING: no knee when the concavity would be empty */
  if (ltr) kd.valid = kd.right < Wp;
  else kd.valid = kd.left > 0;
  return kd;
}

/* Sec. 4.4 "Performance Optimization": the remaining charts folded by a   */
/* prefix sum, then pushed row by row.  The prefix runs over the offsets    */
/* between consecutive charts (padded width minus the compacting distance   */
/* to the next chart; with compaction off, the width), as a recurrence so   */
/* the compacted fold keeps its rule that chart s+1 never starts left of    */
/* chart s-1's right edge.  READING of the row break and the "intermediate */
/* downscaling": a chart whose unwrapped prefix P lies in [rL, (r+1)L)      */
/* starts tail row r at x = P - rL, with L = W' - wmax + 1 (wmax the widest */
/* remaining padded chart), so every chart ends inside the padded atlas     */
/* (x + w' <= L - 1 + wmax = W').  The rows are thus folded to a width      */
/* shortened by the widest chart instead of overflowing and being scaled    */
/* down afterwards: every chart keeps the candidate scale, so the scales of */
/* all charts stay equal and the area-weighted selection of the final scale */
/* reduces to the largest successful candidate.  READING of FastAtlas's      */
/* fixed alternation: one left-to-right row, then two right-to-left rows,   */
/* starting with the first tail row.  Each row is pushed onto the frontline */
/* exactly like a committed row of Algorithm 5 (mirrored charts in a        */
/* right-to-left row, Algorithm 2 when compacting).                          */
typedef struct {
  int on;
  int64_t L;        /* fold width of the tail rows                    */
  int64_t P;        /* unwrapped prefix of the next row's first chart */
  int64_t Pprev;    /* ... of the chart before it                      */
  int64_t Wprev;    /* padded width of the chart before it             */
  int have_prev;    /* a chart precedes the next row in the tail       */
  int rows;         /* tail rows committed                             */
} Tail;

/* One tail row from rowStart: fold, push, commit.  Returns the last chart */
/* of the row; the frontline, placements and the tail state advance.      */
static int tail_row(int n, int rowStart, int row, Tail *t, int hc, const Env *env,
                    const int32_t *dnext, const uint8_t *cannotA, const uint8_t *cannotB,
                    int64_t Wp, int64_t *front, int64_t *X, int64_t *y, int32_t *place) {
  int64_t B = (t->P / t->L) * t->L; /* the row's start in the unwrapped prefix */
  int64_t P = t->P, Pp = t->Pprev, Wpv = t->Wprev;
  int have = t->have_prev;
  int s = rowStart;
  for (; s < n && P < B + t->L; ++s) {
    X[s] = P - B;
    int64_t nx = P + env[s].wp - (hc ? dnext[s] : 0);
    if (hc && have && nx < Pp + Wpv) nx = Pp + Wpv;
    Pp = P;
    Wpv = env[s].wp;
    have = 1;
    P = nx;
  }
  int e = s - 1;
  t->P = P; t->Pprev = Pp; t->Wprev = Wpv; t->have_prev = have;
  int dir = (t->rows % 3 == 0) ? 0 : 1;
  for (int c = rowStart; c <= e; ++c)
    if (dir == 1) X[c] = Wp - X[c] - env[c].wp;
  for (int c = rowStart; c <= e; ++c) {
    y[c] = 0;
    for (int i = 0; i < env[c].wp; ++i) {
      int ti = dir == 0 ? i : env[c].wp - 1 - i;
      y[c] = mx64(y[c], front[X[c] + i] - env[c].top[ti]);
    }
  }
  if (hc) correct_y_offsets(rowStart, e, cannotA, cannotB, y);
  for (int c = rowStart; c <= e; ++c) {
    for (int i = 0; i < env[c].wp; ++i) {
      int ti = dir == 0 ? i : env[c].wp - 1 - i;
      front[X[c] + i] = mx64(front[X[c] + i], y[c] + env[c].bot[ti]);
    }
    place[6 * c + 0] = (int32_t)X[c];
    place[6 * c + 1] = (int32_t)y[c];
    place[6 * c + 2] = dir;
    place[6 * c + 3] = row;
    place[6 * c + 4] = hc;
    place[6 * c + 5] = 2; /* folded by the prefix sum */
  }
  t->rows += 1;
  return e;
}

enum { CFG_FULL = 0, CFG_KNEE = 1 };

/* Placements in sorted order, 6 int32 per chart: x, y, mirror (right-to-left   */
/* row), row index, compacting on in that row, fold (0 atlas width, 1 knee,       */
/* 2 prefix-sum tail).                                                            */
/* stats[0] = rows committed, [1] = knee-folded rows, [2] = knees found,          */
/* [3] = final committed score (max frontline), [4] = charts placed,              */
/* [5] = tail rows (Sec. 4.4).                                                    */
static int pack_scale_env(int n, const Env *env, const int64_t *hq, const int32_t *dnext,
                          const uint8_t *cannotA, const uint8_t *cannotB,
                          int32_t W, int32_t H, const int32_t *params,
                          int32_t *place, int32_t *stats) {
  int g = params[P_GUTTER];
  int flags = params[P_FLAGS];
  int64_t Wp = (int64_t)W + 2 * g, Hp = (int64_t)H + 2 * g;
  int64_t *front = (int64_t *)calloc(Wp, sizeof(int64_t));
  int64_t *local[8], *X[8], *y[8], *pos[2][2];
  for (int j = 0; j < 8; ++j) {
    local[j] = (int64_t *)malloc(sizeof(int64_t) * Wp);
    X[j] = (int64_t *)malloc(sizeof(int64_t) * n);
    y[j] = (int64_t *)malloc(sizeof(int64_t) * n);
  }
  for (int f = 0; f < 2; ++f)
    for (int h = 0; h < 2; ++h) pos[f][h] = (int64_t *)malloc(sizeof(int64_t) * n);
  memset(stats, 0, sizeof(int32_t) * 6);
  /* Sec. 4.4: the hybrid applies to atlases of more than hybrid_min charts */
  /* (the paper: t_opt = 1 % above 10,000 charts, none below).             */
  const int hybrid = params[P_TOPT] > 0 && n > params[P_HYBRID_MIN];
  Tail tail = {0, 1, 0, 0, 0, 0, 0};

  int rowStart = 0, overflow = 0, row = 0;
  int prev_ltr = 0; /* READING: direction ties alternate, the first row left-to-right */
  int64_t committed = 0;
  Knee kd = {0, 1, 0, 0};
  while (rowStart < n && !overflow) {
    /* Sec. 4.4: switch to prefix-sum folding once no knee is live and the  */
    /* row's tallest chart (its first) is below t_opt of the atlas height   */
    /* (READING: its scaled height, without gutters; t_opt in permille).    */
    if (hybrid && !tail.on && !kd.valid &&
        1000 * ((int64_t)env[rowStart].hp - 2 * g) < (int64_t)params[P_TOPT] * H) {
      int64_t wmax = 0;
      for (int s = rowStart; s < n; ++s) wmax = mx64(wmax, env[s].wp);
      if (wmax > Wp) { overflow = 1; break; } /* a chart wider than the atlas */
      tail.on = 1;
      tail.L = Wp - wmax + 1;
    }
    if (tail.on) {
      int hc = (flags & F_HC) != 0;
      int e = tail_row(n, rowStart, row, &tail, hc, env, dnext, cannotA, cannotB, Wp, front, X[0], y[0], place);
      committed = 0;
      for (int64_t xx = 0; xx < Wp; ++xx) committed = mx64(committed, front[xx]);
      overflow = committed > Hp;
      prev_ltr = place[6 * e + 2] == 0;
      stats[4] = e + 1;
      stats[5] = tail.rows;
      rowStart = e + 1;
      ++row;
      continue;
    }
    if (kd.valid) update_knee(&kd, front);
    int nfold = kd.valid ? 2 : 1;
    int rowEnd[2][2];
    int64_t regionLo[2], regionHi[2];
    regionLo[CFG_FULL] = 0;
    regionHi[CFG_FULL] = Wp;
    if (kd.valid) {
      regionLo[CFG_KNEE] = kd.ltr ? kd.right : 0;
      regionHi[CFG_KNEE] = kd.ltr ? Wp : kd.left;
    }
    int nhc = (flags & F_HC) ? 2 : 1;
    for (int f = 0; f < nfold; ++f)
      for (int h = 0; h < 2; ++h)
        rowEnd[f][h] = (h < nhc) ? fold_row(n, rowStart, regionHi[f] - regionLo[f], h, env, dnext, pos[f][h])
                                 : rowStart - 1;
    if (rowEnd[CFG_FULL][0] < rowStart) { overflow = 1; break; } /* a chart wider than the atlas */

    int64_t score[8], scoreKnee[8];
    int valid[8];
    for (int f = 0; f < nfold; ++f)
      for (int h = 0; h < nhc; ++h)
        for (int dir = 0; dir < 2; ++dir) { /* dir 0 = left-to-right, 1 = right-to-left */
          int j = f * 4 + h * 2 + dir;
          valid[j] = rowEnd[f][h] >= rowStart;
          if (!valid[j]) continue;
          int e = rowEnd[f][h];
          for (int s = rowStart; s <= e; ++s)
            X[j][s] = dir == 0 ? regionLo[f] + pos[f][h][s] : regionHi[f] - pos[f][h][s] - env[s].wp;
          /* pushing step: copy the frontline, push each chart to it */
          memcpy(local[j], front, sizeof(int64_t) * Wp);
          for (int s = rowStart; s <= e; ++s) {
            y[j][s] = 0;
            for (int i = 0; i < env[s].wp; ++i) {
              int ti = dir == 0 ? i : env[s].wp - 1 - i; /* a right-to-left row reflects the charts */
              y[j][s] = mx64(y[j][s], local[j][X[j][s] + i] - env[s].top[ti]);
            }
          }
          if (h == 1) correct_y_offsets(rowStart, e, cannotA, cannotB, y[j]);
          for (int s = rowStart; s <= e; ++s)
            for (int i = 0; i < env[s].wp; ++i) {
              int ti = dir == 0 ? i : env[s].wp - 1 - i;
              int64_t xx = X[j][s] + i;
              local[j][xx] = mx64(local[j][xx], y[j][s] + env[s].bot[ti]);
            }
          /* compute score */
          score[j] = 0;
          for (int64_t xx = 0; xx < Wp; ++xx) score[j] = mx64(score[j], local[j][xx]);
          scoreKnee[j] = 0;
          if (f == CFG_KNEE)
            for (int64_t xx = regionLo[f]; xx < regionHi[f]; ++xx)
              scoreKnee[j] = mx64(scoreKnee[j], local[j][xx]);
        }

    /* Sec. 4.2 hierarchical selection.  Level 1: compacting on iff it fits  */
    /* more charts into the row (READING: ties keep it off).  Level 2: the   */
    /* direction with the smaller maximum frontline (whole frontline at the  */
    /* atlas width, the knee concavity when knee-folded); READING: ties go   */
    /* opposite to the previous row.  Level 3: the knee-folded combination   */
    /* wins iff its whole-frontline maximum is smaller by knee_margin.       */
    int choose[2];
    for (int f = 0; f < nfold; ++f) {
      int h = (nhc == 2 && rowEnd[f][1] > rowEnd[f][0]) ? 1 : 0;
      int jl = f * 4 + h * 2 + 0, jr = jl + 1;
      int64_t kl = f == CFG_FULL ? score[jl] : scoreKnee[jl];
      int64_t kr = f == CFG_FULL ? score[jr] : scoreKnee[jr];
      int dir;
      if (flags & F_BALANCE) {
        if (kl < kr) dir = 0;
        else if (kr < kl) dir = 1;
        else dir = prev_ltr ? 1 : 0;
      } else {
        dir = prev_ltr ? 1 : 0; /* static alternation */
      }
      choose[f] = jl + dir;
    }
    int best = choose[CFG_FULL];
    if (nfold == 2 && valid[choose[CFG_KNEE]] &&
        score[choose[CFG_KNEE]] + params[P_KNEE_MARGIN] <= score[best])
      best = choose[CFG_KNEE];
    int bf = best / 4, bh = (best / 2) % 2, bdir = best % 2;
    int e = rowEnd[bf][bh];

    /* commit the best configuration */
    memcpy(front, local[best], sizeof(int64_t) * Wp);
    for (int s = rowStart; s <= e; ++s) {
      place[6 * s + 0] = (int32_t)X[best][s];
      place[6 * s + 1] = (int32_t)y[best][s];
      place[6 * s + 2] = bdir;
      place[6 * s + 3] = row;
      place[6 * s + 4] = bh;
      place[6 * s + 5] = bf;
    }
    if (bf == CFG_FULL) {
      kd = (flags & F_BALANCE) ? find_knee(rowStart, e, bdir == 0, X[best], env, hq, H, (int32_t)Wp, params)
                               : (Knee){0, 1, 0, 0};
      stats[2] += kd.valid;
    } else {
      stats[1] += 1;
    }
    committed = score[best];
    overflow = committed > Hp;
    prev_ltr = bdir == 0;
    stats[4] = e + 1;
    rowStart = e + 1;
    ++row;
  }
  stats[0] = row;
  stats[3] = (int32_t)committed;
  free(front);
  for (int j = 0; j < 8; ++j) { free(local[j]); free(X[j]); free(y[j]); }
  for (int f = 0; f < 2; ++f)
    for (int h = 0; h < 2; ++h) free(pos[f][h]);
  return !overflow && rowStart >= n;
}

/* Envelopes, distances and flags of all sorted charts at scale k. */
typedef struct {
  int n;
  Env *env;
  int32_t *pool;
  int64_t *hq;
  int32_t *dnext;
  uint8_t *cannotA, *cannotB;
} ScaleData;

static int build_scale(int n, const int64_t *rec, const int32_t *perm, int32_t k,
                       const int32_t *params, ScaleData *sd) {
  int g = params[P_GUTTER];
  sd->n = n;
  sd->env = (Env *)calloc(n, sizeof(Env));
  sd->hq = (int64_t *)malloc(sizeof(int64_t) * n);
  sd->dnext = (int32_t *)calloc(n, sizeof(int32_t));
  sd->cannotA = (uint8_t *)calloc(n, 1);
  sd->cannotB = (uint8_t *)calloc(n, 1);
  int64_t total = 0;
  for (int s = 0; s < n; ++s) {
    const int64_t *r = rec + (int64_t)perm[s] * OR_REC;
    total += 2 * (scaled_len(r[R_WQ], k) + 2 * g) + 2 * (scaled_len(r[R_HQ], k) + 2 * g);
  }
  sd->pool = (int32_t *)malloc(sizeof(int32_t) * (total + 1));
  int32_t *p = sd->pool;
  for (int s = 0; s < n; ++s) {
    const int64_t *r = rec + (int64_t)perm[s] * OR_REC;
    int64_t wp = scaled_len(r[R_WQ], k) + 2 * g, hp = scaled_len(r[R_HQ], k) + 2 * g;
    Env *e = &sd->env[s];
    e->top = p; e->bot = p + wp; e->left = p + 2 * wp; e->right = p + 2 * wp + hp;
    p += 2 * wp + 2 * hp;
    int32_t wh[2];
    if (oracle_envelope_padded(r, k, params, wh, e->top, e->bot, e->left, e->right, 1 << 30)) return 1;
    e->wp = wh[0];
    e->hp = wh[1];
    sd->hq[s] = r[R_HQ];
  }
  for (int s = 0; s + 1 < n; ++s) {
    int32_t out[3];
    hcompact_env(sd->env[s].wp, sd->env[s].hp, sd->env[s].right, sd->env[s + 1].hp,
                 sd->env[s + 1].left, out);
    sd->dnext[s] = out[0];
    sd->cannotA[s] = (uint8_t)out[1];
    sd->cannotB[s] = (uint8_t)out[2];
  }
  return 0;
}

static void free_scale(ScaleData *sd) {
  free(sd->env); free(sd->pool); free(sd->hq); free(sd->dnext); free(sd->cannotA); free(sd->cannotB);
}

/* Distances and flags for all adjacent sorted pairs at scale k (for tests). */
int oracle_scale_pairs(int32_t n, const int64_t *rec, const int32_t *perm, int32_t k,
                       const int32_t *params, int32_t *d, uint8_t *cannotA, uint8_t *cannotB,
                       int32_t *wp, int32_t *hp) {
  ScaleData sd;
  if (build_scale(n, rec, perm, k, params, &sd)) { free_scale(&sd); return 1; }
  for (int s = 0; s < n; ++s) {
    d[s] = sd.dnext[s]; cannotA[s] = sd.cannotA[s]; cannotB[s] = sd.cannotB[s];
    wp[s] = sd.env[s].wp; hp[s] = sd.env[s].hp;
  }
  free_scale(&sd);
  return 0;
}

int oracle_pack_scale(int32_t n, const int64_t *rec, const int32_t *perm, int32_t W, int32_t H,
                      int32_t k, const int32_t *params, int32_t *place, int32_t *stats) {
  ScaleData sd;
  if (build_scale(n, rec, perm, k, params, &sd)) { free_scale(&sd); return -1; }
  int ok = pack_scale_env(n, sd.env, sd.hq, sd.dnext, sd.cannotA, sd.cannotB, W, H, params, place, stats);
  free_scale(&sd);
  return ok;
}

/* Literal Algorithm 2 on an explicit offset array (for tests). */
void oracle_correct_y(int32_t s0, int32_t s1, const uint8_t *cannotA, const uint8_t *cannotB,
                      int64_t *y) {
  correct_y_offsets(s0, s1, cannotA, cannotB, y);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1 / Sec. 5 scale search: candidates k = 16j, j = 1..64; the      */
/* largest k whose packing succeeds.  all_scales=1 evaluates every          */
/* candidate (success_per_k[j-1]); otherwise the search runs from the top   */
/* and stops at the first success (same result).                            */
/* place_out (input order, 10 int32 per chart): x, y, rot90, flip_x, flip_y, */
/* mirror, row, sorted position, compacting on, knee-folded.                 */
/* Returns 0 ok, 1 invalid input, 2 no fit.                                  */
/* ------------------------------------------------------------------------ */
int oracle_pack(int32_t n, const uint32_t *offsets, const int32_t *verts, int32_t W, int32_t H,
                const int32_t *params, int32_t all_scales, int32_t *out_k, int32_t *place_out,
                int32_t *success_per_k, int32_t *stats_out) {
  if (W < 1 || H < 1 || W > 8192 || H > 8192) return 1;
  int64_t *rec = (int64_t *)malloc(sizeof(int64_t) * OR_REC * n);
  if (oracle_prep(n, offsets, verts, params, rec)) { free(rec); return 1; }
  int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * n);
  oracle_sort(n, rec, perm);
  int32_t *place = (int32_t *)malloc(sizeof(int32_t) * 6 * n);
  int32_t *best_place = (int32_t *)malloc(sizeof(int32_t) * 6 * n);
  int32_t stats[6], best_stats[6] = {0, 0, 0, 0, 0, 0};
  int best_k = 0;
  for (int j = 64; j >= 1; --j) {
    int32_t k = 16 * j;
    if (!all_scales && best_k) break;
    int ok = oracle_pack_scale(n, rec, perm, W, H, k, params, place, stats);
    if (success_per_k) success_per_k[j - 1] = ok == 1;
    if (ok == 1 && !best_k) {
      best_k = k;
      memcpy(best_place, place, sizeof(int32_t) * 6 * n);
      memcpy(best_stats, stats, sizeof(best_stats));
    }
  }
  *out_k = best_k;
  if (stats_out) memcpy(stats_out, best_stats, sizeof(best_stats));
  if (best_k) {
    for (int s = 0; s < n; ++s) {
      int c = perm[s];
      const int64_t *r = rec + (int64_t)c * OR_REC;
      int32_t *o = place_out + 10 * c;
      o[0] = best_place[6 * s + 0];
      o[1] = best_place[6 * s + 1];
      o[2] = (int32_t)r[R_ROT];
      o[3] = (int32_t)r[R_FLIPX];
      o[4] = (int32_t)r[R_FLIPY];
      o[5] = best_place[6 * s + 2];
      o[6] = best_place[6 * s + 3];
      o[7] = s;
      o[8] = best_place[6 * s + 4];
      o[9] = best_place[6 * s + 5];
    }
  }
  free(rec); free(perm); free(place); free(best_place);
  return best_k ? 0 : 2;
}

int oracle_rec_fields(void) { return OR_REC; }
