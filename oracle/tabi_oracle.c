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
 *             App. A "Computing Oriented Bounding Boxes": 8 angles in
 *             [0, 7pi/16], minimum-area box.
 *   sort      Sec. 3.1: decreasing AABB height.
 *   envelope  App. A "Parallel Pushing Algorithm": TopEdge/BottomEdge per
 *             texel column as the tighter of the two proxies, top rounded
 *             outward, bottom rounded outward; the same per texel row
 *             (left/right extents) for horizontal compaction; Sec. 4.1.1
 *             "merge ... taking the tighter bound": the local-AABB proxy's
 *             bound in a column is the tighter of the x-slices' and the
 *             y-slices' bounds there; Sec. 5 gutters.
 *   hcompact  Sec. 4.1.2 compacting distance; App. A "Detecting Interlocking
 *             Charts" (CannotMoveAbove).
 *   row loop  Algorithm 5 with Algorithm 4 (FoldRow), Algorithm 2
 *             (CorrectYOffsets, the literal do-while), Algorithm 3
 *             (UpdateKneeLocation), knee detection (App. A "Knee Detection
 *             Parameters") and the hierarchical selection of Sec. 4.2.
 *   hybrid    Sec. 4.4: past the rows with knees and tall charts, the rest
 *             of the charts are folded by a prefix sum of their offsets,
 *             downscaled until the overflowing rows fit, and pushed row by
 *             row in a fixed direction pattern.
 *   search    Sec. 3.1 / Sec. 5: 64 candidate scales; Sec. 4.4: the success
 *             with the largest area-weighted mean final scale wins (without
 *             a tail: the largest successful scale).
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
  R_YLO = 37, R_YHI = 47, R_XLO = 57, R_XHI = 67,  /* final slices          */
  R_ATOP = 77, R_ABOT, R_ALEFT, R_ARIGHT, R_ABL2, R_ABR2,
  R_LK = 83            /* K: local AABBs per axis of this record         */
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
/* AABB proxy bounds the column by the x-slices whose open x-interval meets  */
/* it, merged (Sec. 4.1.1, READING: per column, the tighter of the two) with */
/* the bound of the y-slices whose x-range meets it: a chart point in the    */
/* column lies in some y-slice j, so it is no higher than Y_j and no lower   */
/* than Y_j+1 (a per-slice merge instead would change nothing: the slice     */
/* holding an x-slice's topmost point always meets that x-slice).  The OBB   */
/* contributes the minimum (maximum) of its top (bottom)                     */
/* boundary over the column, reached at the box corner when the corner lies  */
/* inside the column and at the nearer column end otherwise (each boundary   */
/* is the max (min) of two lines).  The per-row left/right extents are the   */
/* same construction with the axes swapped.                                  */
/* cols = 0 skips the columns (TopEdge/BottomEdge): the tail's trial scales */
/* need widths and per-row extents only.                                     */
static int envelope_impl(const int64_t *r, int32_t k, const int32_t *params, int32_t *wh,
                         int32_t *top, int32_t *bot, int32_t *left, int32_t *right, int32_t cap, int cols) {
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

  for (int64_t c = 0; c < w && cols; ++c) {
    int64_t a = c * F, b = mn64((c + 1) * F, Wq * k);
    int64_t T = 0, B = h;
    if (use_l) {
      /* the x-slices meeting the column bound its top and bottom by their */
      /* extremes; the y-slices bound them by their own extent: the chart's */
      /* top in the column is no higher than the first y-slice whose        */
      /* x-range meets the column, its bottom no lower than the last one.   */
      /* Sec. 4.1.1's merge keeps the tighter of the two.                   */
      int64_t tl = INT64_MAX, bl = INT64_MIN, t2 = INT64_MAX, b2 = INT64_MIN;
      for (int i = 0; i < K; ++i)
        if (r[R_X + i] * k < b && r[R_X + i + 1] * k > a) {
          tl = mn64(tl, r[R_YLO + i]);
          bl = mx64(bl, r[R_YHI + i]);
        }
      for (int j = 0; j < K; ++j)
        if (r[R_XLO + j] * k < b && r[R_XHI + j] * k > a) {
          t2 = mn64(t2, r[R_Y + j]);
          b2 = mx64(b2, r[R_Y + j + 1]);
        }
      if (t2 != INT64_MAX) { tl = mx64(tl, t2); bl = mn64(bl, b2); }
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
      /* the same with the axes swapped: y-slices bound the row by their   */
      /* extremes, x-slices whose y-range meets the row by their extent    */
      int64_t ll = INT64_MAX, rl = INT64_MIN, l2 = INT64_MAX, r2 = INT64_MIN;
      for (int j = 0; j < K; ++j)
        if (r[R_Y + j] * k < b && r[R_Y + j + 1] * k > a) {
          ll = mn64(ll, r[R_XLO + j]);
          rl = mx64(rl, r[R_XHI + j]);
        }
      for (int i = 0; i < K; ++i)
        if (r[R_YLO + i] * k < b && r[R_YHI + i] * k > a) {
          l2 = mn64(l2, r[R_X + i]);
          r2 = mx64(r2, r[R_X + i + 1]);
        }
      if (l2 != INT64_MAX) { ll = mx64(ll, l2); rl = mn64(rl, r2); }
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

int oracle_envelope(const int64_t *r, int32_t k, const int32_t *params, int32_t *wh,
                    int32_t *top, int32_t *bot, int32_t *left, int32_t *right, int32_t cap) {
  return envelope_impl(r, k, params, wh, top, bot, left, right, cap, 1);
}

/* Sec. 5 gutters (g texels around each chart, none at the atlas edges).     */
/* READING: each envelope is dilated by g in the Chebyshev sense into padded */
/* coordinates (width w+2g, height h+2g); padded footprints must be disjoint */
/* inside the padded atlas (W+2g) x (H+2g).  A chart whose padded footprint  */
/* starts at padded (X, Y) has its texels at atlas (X, Y) onward.            */
static int envelope_padded_impl(const int64_t *r, int32_t k, const int32_t *params, int32_t *wh,
                                int32_t *topP, int32_t *botP, int32_t *leftP, int32_t *rightP,
                                int32_t cap, int cols) {
  int g = params[P_GUTTER];
  int64_t w = scaled_len(r[R_WQ], k), h = scaled_len(r[R_HQ], k);
  if (w > cap || h > cap) { wh[0] = (int32_t)w; wh[1] = (int32_t)h; return 1; }
  int32_t *t = (int32_t *)malloc(sizeof(int32_t) * (w + h + 2));
  int32_t *bo = (int32_t *)malloc(sizeof(int32_t) * (w + 1));
  int32_t *l = (int32_t *)malloc(sizeof(int32_t) * (h + 1));
  int32_t *ri = (int32_t *)malloc(sizeof(int32_t) * (h + 1));
  int32_t whr[2];
  envelope_impl(r, k, params, whr, t, bo, l, ri, cap, cols);
  int64_t wp = w + 2 * g, hp = h + 2 * g;
  wh[0] = (int32_t)wp;
  wh[1] = (int32_t)hp;
  if (wp > cap || hp > cap) { free(t); free(bo); free(l); free(ri); return 1; }
  for (int64_t i = 0; i < wp && cols; ++i) {
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

int oracle_envelope_padded(const int64_t *r, int32_t k, const int32_t *params, int32_t *wh,
                           int32_t *topP, int32_t *botP, int32_t *leftP, int32_t *rightP,
                           int32_t cap) {
  return envelope_padded_impl(r, k, params, wh, topP, botP, leftP, rightP, cap, 1);
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

/* Envelopes, distances and flags of sorted charts at scale k. */
typedef struct {
  int n;
  Env *env;
  int32_t *pool;
  int64_t *hq;
  int32_t *dnext;
  uint8_t *cannotA, *cannotB;
} ScaleData;

static int build_scale(int n, const int64_t *rec, const int32_t *perm, int32_t k,
                       const int32_t *params, ScaleData *sd, int cols);
static void free_scale(ScaleData *sd);

/* x offsets of the charts of one row laid from its near end: Algorithm 4's */
/* recurrence (x of the next chart = x + w' - d with compacting, x + w'     */
/* without; with compacting never left of the right edge of the chart two  */
/* places before, READING 11 of the sequential fold).  x[0..m-1] relative  */
/* to the row's first chart; returns the row's extent max(x + w').          */
static int64_t lay_row(int m, const Env *env, const int32_t *dnext, int hc, int64_t *x) {
  int64_t ext = 0;
  for (int t = 0; t < m; ++t) {
    if (t == 0) x[t] = 0;
    else {
      x[t] = x[t - 1] + env[t - 1].wp - (hc ? dnext[t - 1] : 0);
      if (hc && t >= 2 && x[t] < x[t - 2] + env[t - 2].wp) x[t] = x[t - 2] + env[t - 2].wp;
    }
    ext = mx64(ext, x[t] + env[t].wp);
  }
  return ext;
}

/* Sec. 4.4 "Performance Optimization": once the rows no longer hold knees   */
/* or tall charts, the remaining charts (sorted positions c0..n-1) are laid */
/* out in one pass instead of row by row:                                    */
/*  1. prefix-sum folding at the candidate scale S: the prefix of the        */
/*     offsets between consecutive charts (padded width minus the compacting */
/*     distance to the next chart; the padded width without compacting;     */
/*     READING: the compacted fold keeps its rule that a chart never starts  */
/*     left of the right edge of the chart two places before) puts chart s   */
/*     at P_s, and the rows are cut modulo the padded atlas width: chart s   */
/*     belongs to tail row floor(P_s / W'), so a row's last chart may        */
/*     overflow the width;                                                   */
/*  2. intermediate downscaling: READING (on the k/1024 grid, integer): the  */
/*     tail charts take the largest scale k' in S - 14 .. S at which every  */
/*     tail row, re-laid from its near end with the envelopes, widths and    */
/*     compacting distances at k', fits the padded width W'.  The paper     */
/*     downscales continuously and finds the effect negligible for charts   */
/*     this small; here widths are whole texels with a fixed 2g gutter, so a */
/*     row of one- or two-texel charts can need a large downscale, or none  */
/*     fits.  The tail is therefore taken only when the downscale stays      */
/*     within one step of the candidate grid (15/1024); otherwise nothing   */
/*     is committed and the remaining charts are folded row by row as       */
/*     before the switch (t_opt = 0 for them);                              */
/*  3. the rows, drawn at k', go into the atlas in FastAtlas's fixed         */
/*     alternation (READING: one left-to-right row, then two right-to-left   */
/*     rows, starting with the first tail row) and are pushed up onto the    */
/*     frontline like committed rows of Algorithm 5 (mirrored charts in a    */
/*     right-to-left row, Algorithm 2 when compacting).                      */
/* The tail charts' final scale is k', the others' S; the search then keeps */
/* the candidate whose area-weighted mean final scale is largest.           */
/* Returns 1 if every row fits below the padded height, 0 if one does not,  */
/* -1 if no tail scale fits (nothing placed: the rows continue one by one); */
/* the tail placements go to place (sorted positions), the rows it          */
/* committed and its scale to stats.                                         */
/* Whether every tail row, re-laid at scale k2, fits the padded width. */
static int tail_rows_fit(int m, int nr, const int32_t *rstart, const int64_t *rec, const int32_t *perm,
                         int32_t k2, const int32_t *params, int hc, int64_t Wp, int64_t *x) {
  ScaleData sd;
  int fits = !build_scale(m, rec, perm, k2, params, &sd, 0);
  for (int r = 0; r < nr && fits; ++r) {
    const int a = rstart[r], b = rstart[r + 1];
    fits = lay_row(b - a, sd.env + a, sd.dnext + a, hc, x + a) <= Wp;
  }
  free_scale(&sd);
  return fits;
}

static int tail_pack(int n, int c0, int row, const Env *env, const int32_t *dnext,
                     const int64_t *rec, const int32_t *perm, int32_t S, const int32_t *params,
                     int64_t Wp, int64_t Hp, int64_t *front, int32_t *place, int32_t *stats,
                     int64_t *committed) {
  const int hc = (params[P_FLAGS] & F_HC) != 0;
  const int m = n - c0;
  int64_t *P = (int64_t *)malloc(sizeof(int64_t) * m);
  int32_t *rstart = (int32_t *)malloc(sizeof(int32_t) * (m + 1));
  int64_t *x = (int64_t *)malloc(sizeof(int64_t) * m);
  int64_t *y = (int64_t *)malloc(sizeof(int64_t) * m);

  /* 1. prefix-sum folding at S, rows cut modulo W' */
  for (int t = 0; t < m; ++t) {
    const int s = c0 + t;
    if (t == 0) P[t] = 0;
    else {
      P[t] = P[t - 1] + env[s - 1].wp - (hc ? dnext[s - 1] : 0);
      if (hc && t >= 2 && P[t] < P[t - 2] + env[s - 2].wp) P[t] = P[t - 2] + env[s - 2].wp;
    }
  }
  int nr = 0;
  for (int t = 0; t < m; ++t)
    if (t == 0 || P[t] / Wp != P[t - 1] / Wp) rstart[nr++] = t;
  rstart[nr] = m;

  /* 2. intermediate scale k': the largest of S - 14 .. S at which every */
  /*    row fits, else no tail                                            */
  int32_t kt = 0;
  for (int32_t k2 = S; k2 >= 1 && k2 >= S - 14 && !kt; --k2)
    if (tail_rows_fit(m, nr, rstart, rec, perm + c0, k2, params, hc, Wp, x)) kt = k2;
  if (!kt) {
    free(P); free(rstart); free(x); free(y);
    return -1;
  }
  stats[6] = kt;
  stats[7] = c0;
  ScaleData sd;
  int ok = !build_scale(m, rec, perm + c0, kt, params, &sd, 1);
  for (int r = 0; r < nr && ok; ++r)
    lay_row(rstart[r + 1] - rstart[r], sd.env + rstart[r], sd.dnext + rstart[r], hc, x + rstart[r]);

  /* 3. the rows at k', FastAtlas's directions, pushed onto the frontline */
  for (int r = 0; r < nr && ok; ++r) {
    const int a = rstart[r], b = rstart[r + 1];
    const int dir = (r % 3 == 0) ? 0 : 1;
    const Env *e = sd.env;
    for (int t = a; t < b; ++t) {
      const int64_t X = dir ? Wp - x[t] - e[t].wp : x[t];
      y[t] = 0;
      for (int i = 0; i < e[t].wp; ++i) {
        const int ti = dir == 0 ? i : e[t].wp - 1 - i;
        y[t] = mx64(y[t], front[X + i] - e[t].top[ti]);
      }
      x[t] = X;
    }
    if (hc) correct_y_offsets(a, b - 1, sd.cannotA, sd.cannotB, y);
    for (int t = a; t < b; ++t) {
      for (int i = 0; i < e[t].wp; ++i) {
        const int ti = dir == 0 ? i : e[t].wp - 1 - i;
        front[x[t] + i] = mx64(front[x[t] + i], y[t] + e[t].bot[ti]);
      }
      int32_t *pl = place + 7 * (c0 + t);
      pl[0] = (int32_t)x[t];
      pl[1] = (int32_t)y[t];
      pl[2] = dir;
      pl[3] = row + r;
      pl[4] = hc;
      pl[5] = 2; /* folded by the prefix sum */
      pl[6] = kt;
    }
    *committed = 0;
    for (int64_t xx = 0; xx < Wp; ++xx) *committed = mx64(*committed, front[xx]);
    ok = *committed <= Hp;
    stats[0] = row + r + 1;
    stats[4] = c0 + b;
    stats[5] = r + 1;
  }
  free_scale(&sd);
  free(P); free(rstart); free(x); free(y);
  return ok;
}

enum { CFG_FULL = 0, CFG_KNEE = 1 };

/* Placements in sorted order, 7 int32 per chart: x, y, mirror (right-to-left   */
/* row), row index, compacting on in that row, fold (0 atlas width, 1 knee,       */
/* 2 prefix-sum tail), the chart's scale (S, or the tail's k').                   */
/* stats[0] = rows committed, [1] = knee-folded rows, [2] = knees found,          */
/* [3] = final committed score (max frontline), [4] = charts placed,              */
/* [5] = tail rows, [6] = the tail's scale k' (0: no tail, or none fitted),       */
/* [7] = first tail chart (n: no tail) (Sec. 4.4).                                */
static int pack_scale_env(int n, const Env *env, const int64_t *hq, const int32_t *dnext,
                          const uint8_t *cannotA, const uint8_t *cannotB,
                          int32_t W, int32_t H, const int64_t *rec, const int32_t *perm,
                          int32_t S, const int32_t *params, int32_t *place, int32_t *stats) {
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
  memset(stats, 0, sizeof(int32_t) * 8);
  stats[7] = n;
  /* Sec. 4.4: the hybrid applies to atlases of more than hybrid_min charts */
  /* (the paper: t_opt = 1 % above 10,000 charts, none below).             */
  int hybrid = params[P_TOPT] > 0 && n > params[P_HYBRID_MIN];
  int tail_ok = -1; /* -1: no tail */

  int rowStart = 0, overflow = 0, row = 0;
  int prev_ltr = 0; /* READING: direction ties alternate, the first row left-to-right */
  int64_t committed = 0;
  Knee kd = {0, 1, 0, 0};
  while (rowStart < n && !overflow) {
    /* Sec. 4.4: switch to prefix-sum folding once no knee is live and the  */
    /* row's tallest chart (its first) is below t_opt of the atlas height   */
    /* (READING: its scaled height, without gutters; t_opt in permille).    */
    if (hybrid && !kd.valid &&
        1000 * ((int64_t)env[rowStart].hp - 2 * g) < (int64_t)params[P_TOPT] * H) {
      stats[0] = row;
      tail_ok = tail_pack(n, rowStart, row, env, dnext, rec, perm, S, params, Wp, Hp, front, place, stats,
                          &committed);
      if (tail_ok >= 0) {
        row = stats[0];
        rowStart = stats[4];
        break;
      }
      hybrid = 0; /* no tail scale within one grid step: the rows go on one by one */
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
      place[7 * s + 0] = (int32_t)X[best][s];
      place[7 * s + 1] = (int32_t)y[best][s];
      place[7 * s + 2] = bdir;
      place[7 * s + 3] = row;
      place[7 * s + 4] = bh;
      place[7 * s + 5] = bf;
      place[7 * s + 6] = S;
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
  if (tail_ok == 0) overflow = 1;
  free(front);
  for (int j = 0; j < 8; ++j) { free(local[j]); free(X[j]); free(y[j]); }
  for (int f = 0; f < 2; ++f)
    for (int h = 0; h < 2; ++h) free(pos[f][h]);
  return !overflow && rowStart >= n;
}

/* Envelopes, distances and flags of the sorted charts perm[0..n-1] at */
/* scale k.                                                              */
static int build_scale(int n, const int64_t *rec, const int32_t *perm, int32_t k,
                       const int32_t *params, ScaleData *sd, int cols) {
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
    if (envelope_padded_impl(r, k, params, wh, e->top, e->bot, e->left, e->right, 1 << 30, cols)) return 1;
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
  if (build_scale(n, rec, perm, k, params, &sd, 1)) { free_scale(&sd); return 1; }
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
  if (build_scale(n, rec, perm, k, params, &sd, 1)) { free_scale(&sd); return -1; }
  int ok = pack_scale_env(n, sd.env, sd.hq, sd.dnext, sd.cannotA, sd.cannotB, W, H, rec, perm, k, params,
                          place, stats);
  free_scale(&sd);
  return ok;
}

/* Literal Algorithm 2 on an explicit offset array (for tests). */
void oracle_correct_y(int32_t s0, int32_t s1, const uint8_t *cannotA, const uint8_t *cannotB,
                      int64_t *y) {
  correct_y_offsets(s0, s1, cannotA, cannotB, y);
}

/* Twice the area of a chart's vertex loop (shoelace), in Q.8^2 units, as */
/* a magnitude: the weight of the chart in the area-weighted mean scale.   */
static int64_t loop_area2(int nv, const int32_t *v) {
  int64_t a2 = 0;
  for (int i = 0; i < nv; ++i) {
    int j = (i + 1) % nv;
    a2 += (int64_t)v[2 * i] * v[2 * j + 1] - (int64_t)v[2 * j] * v[2 * i + 1];
  }
  return a2 < 0 ? -a2 : a2;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1 / Sec. 5 scale search over the candidates S = 16j, j = 1..64,   */
/* with Sec. 4.4's choice: the successful candidate whose mean final scale, */
/* weighted by chart area, is largest -- i.e. the largest                   */
/* sum_c area_c * scale_c (scale_c = S, or k' for the prefix-sum tail's     */
/* charts), compared exactly; READING: ties keep the larger S.  Without a   */
/* tail every chart has scale S and this is the largest successful S.  The */
/* candidates are tried from the top; once one has succeeded, a smaller S   */
/* can only win if S * sum_c area_c exceeds the best sum (no chart's scale  */
/* exceeds its candidate), so the search stops at the first S where it     */
/* does not (all_scales = 1 evaluates every candidate instead, with the     */
/* same result; success_per_k[j-1] records each).                           */
/* place_out (input order, 11 int32 per chart): x, y, rot90, flip_x,         */
/* flip_y, mirror, row, sorted position, compacting on, fold (0 atlas       */
/* width, 1 knee, 2 prefix-sum tail), the chart's scale k.                  */
/* stats_out: the chosen candidate's stats (8, see pack_scale_env), then    */
/* its area-weighted scale sum as two int64 halves (low, high).             */
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
  int64_t *area = (int64_t *)malloc(sizeof(int64_t) * n); /* sorted order */
  i128 area_total = 0;
  for (int s = 0; s < n; ++s) {
    int c = perm[s];
    area[s] = loop_area2((int)(offsets[c + 1] - offsets[c]), verts + 2 * offsets[c]);
    area_total += area[s];
  }
  int32_t *place = (int32_t *)malloc(sizeof(int32_t) * 7 * n);
  int32_t *best_place = (int32_t *)malloc(sizeof(int32_t) * 7 * n);
  int32_t stats[8], best_stats[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int best_k = 0;
  i128 best_score = 0;
  for (int j = 64; j >= 1; --j) {
    int32_t k = 16 * j;
    if (!all_scales && best_k && (i128)k * area_total <= best_score) break;
    int ok = oracle_pack_scale(n, rec, perm, W, H, k, params, place, stats);
    if (success_per_k) success_per_k[j - 1] = ok == 1;
    if (ok != 1) continue;
    i128 score = 0;
    for (int s = 0; s < n; ++s) score += (i128)area[s] * place[7 * s + 6];
    if (!best_k || score > best_score) {
      best_k = k;
      best_score = score;
      memcpy(best_place, place, sizeof(int32_t) * 7 * n);
      memcpy(best_stats, stats, sizeof(best_stats));
    }
  }
  *out_k = best_k;
  if (stats_out) {
    memcpy(stats_out, best_stats, sizeof(best_stats));
    int64_t lo = (int64_t)(uint64_t)best_score, hi = (int64_t)(best_score >> 64);
    memcpy(stats_out + 8, &lo, 8);
    memcpy(stats_out + 10, &hi, 8);
  }
  if (best_k) {
    for (int s = 0; s < n; ++s) {
      int c = perm[s];
      const int64_t *r = rec + (int64_t)c * OR_REC;
      int32_t *o = place_out + 11 * c;
      o[0] = best_place[7 * s + 0];
      o[1] = best_place[7 * s + 1];
      o[2] = (int32_t)r[R_ROT];
      o[3] = (int32_t)r[R_FLIPX];
      o[4] = (int32_t)r[R_FLIPY];
      o[5] = best_place[7 * s + 2];
      o[6] = best_place[7 * s + 3];
      o[7] = s;
      o[8] = best_place[7 * s + 4];
      o[9] = best_place[7 * s + 5];
      o[10] = best_place[7 * s + 6];
    }
  }
  free(rec); free(perm); free(area); free(place); free(best_place);
  return best_k ? 0 : 2;
}

/* Twice the area of every chart's loop, input order: the weights of the  */
/* area-weighted mean scale above.                                          */
void oracle_chart_area2(int32_t n, const uint32_t *offsets, const int32_t *verts, int64_t *out) {
  for (int c = 0; c < n; ++c)
    out[c] = loop_area2((int)(offsets[c + 1] - offsets[c]), verts + 2 * offsets[c]);
}

int oracle_rec_fields(void) { return OR_REC; }
