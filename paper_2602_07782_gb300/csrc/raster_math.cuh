// Per-scanline envelope arithmetic of the rasterizer (App. A "Parallel
// Pushing Algorithm"), shared by the raster kernel and usable on the host.
//
// A scanline is a texel column (axis 0: TopEdge/BottomEdge over x in
// (cF, (c+1)F)) or a texel row (axis 1: left/right extents over y), in
// scaled units (F = 2^18 per texel, scaled coordinate = Q.8 * k).
//
// OBB boundaries.  Each side of the box is the max (or min) of two lines.
// With generic constants (A1, A2, B1, B2 scaled by k; b1, b2 the line
// slopes' numerators; d1, d2 their denominators, all from C_m, S_m):
//   lower(X) = max( floor((A1 - X b1) / (d1 F)), floor((A2 + X b2) / (d2 F)) )
//   upper(X) = min( -floor((B1 + X b1) / (d1 F)), -floor((B2 - X b2) / (d2 F)) )
//   axis 0: A1 = U0, b1 = C, d1 = S, A2 = V0, b2 = S, d2 = C, B1 = -U1, B2 = -V1
//   axis 1: A1 = U0, b1 = S, d1 = C, A2 = -V1, b2 = C, d2 = S, B1 = -U1, B2 = V0
// At a scanline boundary X = cF the F cancels:  floor((A - c b F)/(d F)) =
// floor((floor(A / F) - c b) / d), because adding the remainder (a fraction
// in [0, 1)) to an integer numerator never changes a floor by a positive
// integer d.  All such numerators fit 32 bits (|A|/F < 2^28, c b < 2^27), so
// the per-scanline work is 32-bit; a scanline clipped by the chart's end
// (X = ext * k, not a multiple of F) forms its numerator in 64 bits once per
// candidate and shifts it down first (floor(N / (d F)) = floor(floor(N / F)
// / d)).
// Lower is convex and upper concave in X, so over [a, b] each reaches its
// extreme at the box corner when the corner lies in [a, b], else at the
// nearer end; the corner's position is kept as floor/ceil(pos / N),
// N = C^2 + S^2, which decides both tests exactly for integer a, b, and is
// turned into a range of scanline indices once per candidate.
//
// The 32-bit floor division by d (= C or S, 3196..16384, fixed per angle)
// is a multiply-high by d's magic number and a shift (division by an
// invariant integer, see fdiv_magic), exact for the numerators here
// (|numerator| < 2^29).
//
// Corner values and positions are linear in k: floor(k num / D).  A warp
// that walks the candidates k, k+16, ... keeps (q, r) with k num = q D + r,
// 0 <= r < D, and adds the precomputed (floor(16 num / D), 16 num mod D),
// carrying one when r overflows -- no division per candidate.
#pragma once

#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define TABI_HD __host__ __device__ __forceinline__
#else
#define TABI_HD inline
// host builds (the division tests) get CUDA's 4-int vector by hand
struct int4 {
  int x, y, z, w;
};
inline int4 make_int4(int x, int y, int z, int w) { return int4{x, y, z, w}; }
#endif

namespace tabi {
namespace rmath {

constexpr int kK = 10;
constexpr int64_t kF = 1LL << 18;
constexpr int32_t kInf = 0x3fffffff;

// Division by an invariant integer d by multiplication (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994,
// Thm. 4.2 with N = 31): for 2^(l-1) < d <= 2^l and M = ceil(2^(31+l) / d),
// floor(x / d) = floor(M x / 2^(31+l)) for every 0 <= x < 2^31, and
// M < 2^32.  A numerator |a| < 2^29 is shifted into that range by adding
// B d with B = ceil(2^29 / d), and B is taken off the quotient.
struct Magic {
  uint32_t M;
  int32_t shift;  // l - 1 (the multiply-high already drops 32 bits)
  int32_t bd;     // B d
  int32_t B;
};
constexpr Magic magic_div(uint32_t d) {
  int l = 0;
  while ((1u << l) < d) ++l;
  const uint64_t M = ((1ull << (31 + l)) + d - 1) / d;
  const uint32_t B = ((1u << 29) + d - 1) / d;
  return Magic{(uint32_t)M, l - 1, (int32_t)(B * d), (int32_t)B};
}
TABI_HD uint32_t umulhi32(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}
// floor(a / d) for |a| < 2^29 and the magic numbers of d (d >= 2)
TABI_HD int32_t fdiv_magic(int32_t a, const Magic &mg) {
  return (int32_t)(umulhi32(mg.M, (uint32_t)(a + mg.bd)) >> mg.shift) - mg.B;
}

struct AxisK {
  // local-AABB pieces: first scanline, span (last - first), scaled bounds
  // lo, hi -- one 16-byte record each, so a scanline tests a piece with one
  // broadcast vector load, one unsigned compare and two min/max.  piece[]
  // are the slices along this axis (bounded by their extremes), cross[] the
  // slices along the other axis, whose extent on this axis bounds the
  // scanlines they meet by their own boundaries (Sec. 4.1.1's merge keeps
  // the tighter of the two)
  int4 piece[kK];
  int4 cross[kK];
  // OBB, fast path (X = multiple of F)
  int32_t ah1, ah2, bh1, bh2;   // floor(A1/F), floor(A2/F), floor(B1/F), floor(B2/F)
  int32_t b1, b2, d1, d2;
  Magic q1, q2;                 // exact division by d1, d2 (multiply-high)
  int32_t corner_lo, corner_hi; // extreme values at the corners
  int32_t len, len_other, use_l, use_o;
  // corner tests in scanline units (see corner_store): the corner value
  // applies on scanlines [c0, c1]; scanlines c > f lie wholly past the
  // corner (the bound's extreme over them is at their start)
  int32_t lo_c0, lo_c1, lo_f, hi_c0, hi_c1, hi_f;
  int32_t clip_c;                      // the scanline cut by the chart's end (-1: none)
  int32_t cl_n1, cl_n2, cu_n1, cu_n2;  // shifted numerators at X = end (lower, upper)
  int64_t end;                         // ext * k
  int64_t A1, A2, B1, B2;              // 64-bit form for the clipped scanline
};

TABI_HD int64_t fdiv64(int64_t a, int64_t b) {  // floor, b > 0
  int64_t q = a / b;
  if ((a % b) != 0 && a < 0) --q;
  return q;
}
// floor(a / d) for d > 0, |a| < 2^62, |a / d| < 2^40: the double quotient
// is within 2^-11 of the true one, so its floor is off by at most one and
// the exact remainder a - q d fixes it.
TABI_HD int64_t fdiv64_est(int64_t a, int64_t d) {
  int64_t q = (int64_t)floor((double)a / (double)d);
  const int64_t r = a - q * d;
  if (r < 0) --q;
  else if (r >= d) ++q;
  return q;
}
TABI_HD int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }
TABI_HD int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }
TABI_HD int32_t imin32(int32_t a, int32_t b) { return a < b ? a : b; }
TABI_HD int32_t imax32(int32_t a, int32_t b) { return a > b ? a : b; }

// floor(a / d) for |a| < 2^30, 1 <= d < 2^15, rcp ~ 1/d (float)
TABI_HD int32_t fdiv32(int32_t a, int32_t d, float rcp) {
  int32_t q = (int32_t)floorf((float)a * rcp);
  const int32_t r = a - q * d;
  if (r < 0) --q;
  else if (r >= d) ++q;
  return q;
}

// Local-AABB piece i of an axis at scale k, from its slice bounds
// b0 = floor(i ext / K), b1 = floor((i + 1) ext / K) (ext = Wq or Hq) and
// the slice's extremes lo_q8, hi_q8 on the other axis (ylo/yhi or
// xlo/xhi), all in [0, 2^21): the scaled values stay below 2^31
// (k <= 1024), so 32-bit unsigned arithmetic is exact.
TABI_HD void setup_piece(AxisK &ak, int i, uint32_t b0, uint32_t b1, uint32_t k, uint32_t lo_q8, uint32_t hi_q8) {
  const uint32_t s0 = b0 * k, s1 = b1 * k;
  const int32_t plo = (int32_t)(s0 >> 18);                 // floor(s0 / F)
  const int32_t phi = (int32_t)((s1 + kF - 1) >> 18) - 1;   // ceil(s1 / F) - 1 (>= plo: s1 > s0)
  const int32_t lo = (int32_t)((lo_q8 * k) >> 18);
  const int32_t hi = (int32_t)((hi_q8 * k + kF - 1) >> 18);
  ak.piece[i] = make_int4(plo, phi - plo, lo, hi);
}

// Cross piece i of an axis at scale k: a slice of the other axis, whose
// extent on this axis is [e0, e1] (xlo/xhi of a y-slice for columns,
// ylo/yhi of an x-slice for rows) and whose own boundaries are b0, b1
// (Y_i, Y_i+1 or X_i, X_i+1), all Q.8 in [0, 2^21].  It meets scanline c
// (the open interval (cF, min((c+1)F, end))) iff e0 k < min((c+1)F, end)
// and e1 k > cF, i.e. for floor(e0 k / F) <= c <= ceil(e1 k / F) - 1 when
// e0 < ext (never otherwise: such a slice only touches the far end); on
// them the chart lies between floor(b0 k / F) and ceil(b1 k / F).
TABI_HD void setup_cross(AxisK &ak, int i, uint32_t e0, uint32_t e1, uint32_t ext, uint32_t k, uint32_t b0,
                         uint32_t b1) {
  const int32_t plo = (int32_t)((e0 * k) >> 18);
  const int32_t phi = (int32_t)((e1 * k + kF - 1) >> 18) - 1;
  const int32_t lo = (int32_t)((b0 * k) >> 18);
  const int32_t hi = (int32_t)((b1 * k + kF - 1) >> 18);
  ak.cross[i] = (e0 < ext && phi >= plo) ? make_int4(plo, phi - plo, lo, hi) : make_int4(kInf, 0, lo, hi);
}

// OBB terms of one axis that do not depend on the scale (once per chart).
TABI_HD void setup_obb_fixed(AxisK &ak, int axis, int m, int64_t C, int64_t S, const Magic &qC,
                             const Magic &qS, bool use_l, bool use_o) {
  ak.use_l = use_l;
  ak.use_o = use_o && m > 0;
  if (axis == 0) {
    ak.b1 = (int32_t)C; ak.d1 = (int32_t)S; ak.b2 = (int32_t)S; ak.d2 = (int32_t)C;
  } else {
    ak.b1 = (int32_t)S; ak.d1 = (int32_t)C; ak.b2 = (int32_t)C; ak.d2 = (int32_t)S;
  }
  ak.q1 = axis == 0 ? qS : qC;  // division by d1, d2
  ak.q2 = axis == 0 ? qC : qS;
}

// OBB line terms and scanline counts of one axis at scale k (after
// setup_obb_fixed for the same axis and chart).
TABI_HD void setup_obb_k(AxisK &ak, int axis, int64_t Wq, int64_t Hq, int64_t k, int64_t C, int64_t S,
                         int64_t u0, int64_t u1, int64_t v0, int64_t v1) {
  const int64_t w = (Wq * k + kF - 1) >> 18, h = (Hq * k + kF - 1) >> 18;
  ak.len = (int32_t)(axis == 0 ? w : h);
  ak.len_other = (int32_t)(axis == 0 ? h : w);
  const int64_t end = (axis == 0 ? Wq : Hq) * k;
  ak.end = end;
  ak.clip_c = (end & (kF - 1)) ? ak.len - 1 : -1;
  if (!ak.use_o) return;
  const int64_t U0 = u0 * k, U1 = u1 * k, V0 = v0 * k, V1 = v1 * k;
  const int64_t A1 = U0, A2 = axis == 0 ? V0 : -V1, B1 = -U1, B2 = axis == 0 ? -V1 : V0;
  const int64_t b1 = axis == 0 ? C : S, b2 = axis == 0 ? S : C;
  ak.A1 = A1; ak.A2 = A2; ak.B1 = B1; ak.B2 = B2;
  ak.ah1 = (int32_t)(A1 >> 18); ak.ah2 = (int32_t)(A2 >> 18);
  ak.bh1 = (int32_t)(B1 >> 18); ak.bh2 = (int32_t)(B2 >> 18);
  // at X = end: floor(N / (d F)) = floor(floor(N / F) / d), |N| < 2^47
  ak.cl_n1 = (int32_t)((A1 - end * b1) >> 18);
  ak.cl_n2 = (int32_t)((A2 + end * b2) >> 18);
  ak.cu_n1 = (int32_t)((B1 + end * b1) >> 18);
  ak.cu_n2 = (int32_t)((B2 - end * b2) >> 18);
}

// The eight corner quantities (item = axis * 4 + {0: lower value, 1: upper
// value, 2: lower position, 3: upper position}): floor(k num / D) with
//   lower value  num = (axis 0) u0 S + v0 C,  (axis 1) u0 C - v1 S,  D = N F
//   upper value  num = -((axis 0) u1 S + v1 C, (axis 1) u1 C - v0 S), negated back
//   lower position num = (axis 0) u0 C - v0 S, (axis 1) u0 S + v1 C,  D = N
//   upper position num = (axis 0) u1 C - v1 S, (axis 1) u1 S + v0 C,  D = N
// over the candidates k = 16 (j + 1): from the quotient and remainder of
// one step (16 num = qs D + rs, 0 <= rs < D) a run of candidates starts
// with a small division and then advances by one step per candidate.
struct CornerQ {
  int64_t D, q, r, qs, rs;
};

TABI_HD int64_t corner_num(int item, int64_t C, int64_t S, int64_t u0, int64_t u1, int64_t v0, int64_t v1) {
  const int axis = item >> 2;
  switch (item & 3) {
    case 0: return axis == 0 ? u0 * S + v0 * C : u0 * C - v1 * S;
    case 1: return -(axis == 0 ? u1 * S + v1 * C : u1 * C - v0 * S);
    case 2: return axis == 0 ? u0 * C - v0 * S : u0 * S + v1 * C;
    default: return axis == 0 ? u1 * C - v1 * S : u1 * S + v0 * C;
  }
}
TABI_HD int64_t corner_den(int item, int64_t C, int64_t S) {
  const int64_t N = C * C + S * S;
  return (item & 3) < 2 ? N * kF : N;
}

// floor(a / N) for |a| < 2^62 and 2^23 < N < 2^30 in single precision and
// exact integer corrections.  A float quotient has relative error below
// 2^-22 (three roundings of 2^-24), so the first estimate q1 (|a / N| <
// 2^39) is within 2^17 + 1 of a / N; the remainder a - q1 N is then below
// 2^48 in size, and the estimate of its quotient (below 2^17 + 1) is within
// 2^-5 of the true one, so the sum is off by at most one, which the exact
// remainder fixes.
TABI_HD int64_t fdiv_n(int64_t a, int64_t N) {
  const float rn = 1.0f / (float)N;
  int64_t q = (int64_t)((float)a * rn);
  q += (int64_t)floorf((float)(a - q * N) * rn);
  const int64_t r = a - q * N;
  if (r < 0) --q;
  else if (r >= N) ++q;
  return q;
}

// One step's quotient and remainder.  D = N F or N with N = C^2 + S^2 in
// (2^23, 2^29] and |16 num| < 2^55; floor(a / (N F)) = floor(floor(a / F) / N).
TABI_HD void corner_step(int item, int64_t C, int64_t S, int64_t u0, int64_t u1, int64_t v0, int64_t v1,
                         int64_t &qs, int64_t &rs) {
  const int64_t num = 16 * corner_num(item, C, S, u0, u1, v0, v1);
  const int64_t N = C * C + S * S;
  qs = fdiv_n((item & 3) < 2 ? (num >> 18) : num, N);
  rs = num - qs * corner_den(item, C, S);
}

// Candidate j0 from the step: k0 num = (j0 + 1)(qs D + rs), so
// q = (j0 + 1) qs + floor(t / D) with t = (j0 + 1) rs in [0, 64 D).  The
// float quotient of t / D is below 64 and within 2^-16 of the true one
// (three roundings of relative size 2^-24), so its floor is off by at most
// one and the exact remainder fixes it.
TABI_HD void corner_init(CornerQ &cq, int item, int j0, int64_t C, int64_t S, int64_t qs, int64_t rs) {
  cq.D = corner_den(item, C, S);
  cq.qs = qs;
  cq.rs = rs;
  const int64_t t = (int64_t)(j0 + 1) * rs;
  int64_t qq = (int64_t)floorf((float)t / (float)cq.D);
  int64_t r = t - qq * cq.D;
  if (r < 0) { --qq; r += cq.D; }
  else if (r >= cq.D) { ++qq; r -= cq.D; }
  cq.q = (int64_t)(j0 + 1) * qs + qq;
  cq.r = r;
}

// The same quantity at any scale k <= 1024 directly: k num (|k num| <
// 2^61) divided by D, with the remainder (only its being non-zero is used,
// for the positions).
TABI_HD void corner_at(CornerQ &cq, int item, int64_t k, int64_t C, int64_t S, int64_t u0, int64_t u1,
                       int64_t v0, int64_t v1) {
  const int64_t a = k * corner_num(item, C, S, u0, u1, v0, v1);
  const int64_t N = C * C + S * S;
  cq.D = corner_den(item, C, S);
  cq.qs = cq.rs = 0;
  if ((item & 3) < 2) {
    cq.q = fdiv_n(a >> 18, N);  // floor(a / (N F)) = floor(floor(a / F) / N)
    cq.r = 0;
  } else {
    cq.q = fdiv_n(a, N);
    cq.r = a - cq.q * N;
  }
}

TABI_HD void corner_advance(CornerQ &cq) {
  cq.q += cq.qs;
  cq.r += cq.rs;
  if (cq.r >= cq.D) { cq.r -= cq.D; cq.q += 1; }
}

// Corner position pos (scaled units) as scanline tests.  Over scanline c,
// X in [a, b] = [cF, min((c+1)F, end)], the corner value applies iff
// a <= floor(pos) and ceil(pos) <= b, i.e. iff c0 <= c <= c1 with
// c0 = ceil(ceil(pos)/F) - 1, c1 = floor(floor(pos)/F) when 0 <= pos and
// ceil(pos) <= end, and never otherwise; the scanline lies wholly past the
// corner (floor(pos) < a) iff c > f = floor(floor(pos)/F).
TABI_HD void corner_range(int64_t pf, int64_t pc, int64_t end, int32_t &c0, int32_t &c1, int32_t &f) {
  f = (int32_t)(pf >> 18);
  if (pf < 0 || pc > end) {
    c0 = 1;
    c1 = 0;
  } else {
    c0 = (int32_t)(((pc + kF - 1) >> 18) - 1);
    c1 = f;
  }
}

// Store the corner quantity into its axis' constants.  `end` = ext * k of
// the item's axis.
TABI_HD void corner_store(const CornerQ &cq, int item, AxisK &ak, int64_t end) {
  switch (item & 3) {
    case 0: ak.corner_lo = (int32_t)cq.q; break;
    case 1: ak.corner_hi = (int32_t)-cq.q; break;
    case 2: corner_range(cq.q, cq.q + (cq.r != 0), end, ak.lo_c0, ak.lo_c1, ak.lo_f); break;
    default: corner_range(cq.q, cq.q + (cq.r != 0), end, ak.hi_c0, ak.hi_c1, ak.hi_f); break;
  }
}

// Lower / upper OBB bound at X = q F or, for the scanline cut by the
// chart's end, X = end (the precomputed shifted numerators; both cases take
// the 32-bit division, the shifted numerators being below 2^29).
TABI_HD int32_t obb_lower_at(const AxisK &ak, int32_t q, bool clipped) {
  const int32_t n1 = clipped ? ak.cl_n1 : ak.ah1 - q * ak.b1;
  const int32_t n2 = clipped ? ak.cl_n2 : ak.ah2 + q * ak.b2;
  return imax32(fdiv_magic(n1, ak.q1), fdiv_magic(n2, ak.q2));
}
TABI_HD int32_t obb_upper_at(const AxisK &ak, int32_t q, bool clipped) {
  const int32_t n1 = clipped ? ak.cu_n1 : ak.bh1 + q * ak.b1;
  const int32_t n2 = clipped ? ak.cu_n2 : ak.bh2 - q * ak.b2;
  return imin32(-fdiv_magic(n1, ak.q1), -fdiv_magic(n2, ak.q2));
}

// Raw bounds of scanline c (0 <= c < len): [lo, hi) with hi > lo, given
// the local-AABB bounds pl, ph of the pieces that meet the scanline.
TABI_HD void scanline_from(const AxisK &ak, int32_t c, int32_t pl, int32_t ph, int32_t &lo_out,
                           int32_t &hi_out) {
  int32_t lo = 0, hi = ak.len_other;
  if (ak.use_l) {
    lo = imax32(lo, pl);
    hi = imin32(hi, ph);
  }
  if (ak.use_o) {
    // without branches (the lanes of a chunk straddle the corners): the
    // extreme over the scanline is at its start if the corner lies before
    // it, else at its end (X = end if cut); the corner value if inside
    const bool clip = c == ak.clip_c;
    const bool past_l = c > ak.lo_f, past_h = c > ak.hi_f;
    int32_t tl = obb_lower_at(ak, past_l ? c : c + 1, !past_l && clip);
    int32_t th = obb_upper_at(ak, past_h ? c : c + 1, !past_h && clip);
    tl = (ak.lo_c0 <= c && c <= ak.lo_c1) ? ak.corner_lo : tl;
    th = (ak.hi_c0 <= c && c <= ak.hi_c1) ? ak.corner_hi : th;
    lo = imax32(lo, tl);
    hi = imin32(hi, th);
  }
  lo = imax32(0, imin32(lo, ak.len_other - 1));
  hi = imax32(lo + 1, imin32(hi, ak.len_other));
  lo_out = lo;
  hi_out = hi;
}

// The same with the pieces tested here (all ten per scanline, then the
// ten cross pieces: the tighter of the two bounds).  Some cross piece meets
// every scanline of a valid chart (the chart's boundary crosses every
// scanline and each of its points lies in some slice), which the guard
// only makes explicit.
TABI_HD void scanline(const AxisK &ak, int32_t c, int32_t &lo_out, int32_t &hi_out) {
  int32_t pl = kInf, ph = -kInf;
#pragma unroll
  for (int i = 0; i < kK; ++i) {
    const int4 pc = ak.piece[i];
    if ((uint32_t)(c - pc.x) <= (uint32_t)pc.y) {  // plo <= c <= plo + span
      pl = imin32(pl, pc.z);
      ph = imax32(ph, pc.w);
    }
  }
  if (ak.use_l) {
    int32_t ql = kInf, qh = -kInf;
#pragma unroll
    for (int i = 0; i < kK; ++i) {
      const int4 pc = ak.cross[i];
      if ((uint32_t)(c - pc.x) <= (uint32_t)pc.y) {
        ql = imin32(ql, pc.z);
        qh = imax32(qh, pc.w);
      }
    }
    if (ql != kInf) {
      pl = imax32(pl, ql);
      ph = imin32(ph, qh);
    }
  }
  scanline_from(ak, c, pl, ph, lo_out, hi_out);
}

}  // namespace rmath
}  // namespace tabi
