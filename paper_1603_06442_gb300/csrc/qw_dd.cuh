// Double-double arithmetic for the complex128 eigenphase omega_k.
//
// A double-double is an unevaluated sum hi + lo of FP64 numbers (|lo| <= ulp(hi) / 2,
// about 106 significant bits), kept by error-free transformations: Knuth's two-sum,
// Dekker's fast two-sum (for |a| >= |b|) and the FMA two-product.  The _rn
// intrinsics keep the compiler from contracting or reordering them.
//
// omega_k = atan2(S, C) with S = sqrt(m^2 + n^2 |n~_k|^2), C = n u_k (Sec. 3.2,
// cos omega_k = n u_k) is formed to ~1e-31: the symbol from double-double cos/sin
// of the exact grid angles 2 pi q / P (integer octant reduction, then the Taylor
// series on [0, pi/4]), S by a Newton step on the FP64 square root, and
// omega = theta_j + asin(x) with theta_j = j pi / 1024 the anchor nearest to the
// FP64 atan2 and x = S cos theta_j - C sin theta_j = sin(omega - theta_j),
// |x| < 1.6e-3, whose arcsine series is truncated below 1e-32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qw {

struct dd {
  double hi, lo;
};

__device__ __forceinline__ dd dd_two_sum(double a, double b) {
  const double s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  return dd{s, __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb))};
}
__device__ __forceinline__ dd dd_fast(double a, double b) {  // |a| >= |b|
  const double s = __dadd_rn(a, b);
  return dd{s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ __forceinline__ dd dd_two_prod(double a, double b) {
  const double p = __dmul_rn(a, b);
  return dd{p, __fma_rn(a, b, -p)};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = dd_two_sum(a.hi, b.hi);
  const dd t = dd_two_sum(a.lo, b.lo);
  s = dd_fast(s.hi, __dadd_rn(s.lo, t.hi));
  return dd_fast(s.hi, __dadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const dd p = dd_two_prod(a.hi, b.hi);
  const double c = __fma_rn(a.hi, b.lo, __dmul_rn(a.lo, b.hi));
  return dd_fast(p.hi, __dadd_rn(p.lo, c));
}
__device__ __forceinline__ dd dd_mul_d(dd a, double b) {
  const dd p = dd_two_prod(a.hi, b);
  return dd_fast(p.hi, __fma_rn(a.lo, b, p.lo));
}
__device__ __forceinline__ dd dd_div_d(dd a, double b) {  // a / b
  const double q1 = __ddiv_rn(a.hi, b);
  const dd p = dd_two_prod(q1, b);
  const double r = __dadd_rn(__dsub_rn(__dsub_rn(a.hi, p.hi), p.lo), a.lo);
  return dd_fast(q1, __ddiv_rn(r, b));
}
__device__ __forceinline__ dd dd_sqrt(dd a) {  // a >= 0
  if (!(a.hi > 0.0)) return dd{0.0, 0.0};
  const double s = __dsqrt_rn(a.hi);
  const dd e = dd_sub(a, dd_two_prod(s, s));
  return dd_fast(s, __ddiv_rn(e.hi, 2.0 * s));
}

// pi and pi / 4 as double-double (the exact value's nearest FP64 number plus the
// nearest FP64 number to the remainder)
__device__ __forceinline__ dd dd_pi() { return dd{3.141592653589793116e+00, 1.2246467991473532e-16}; }
__device__ __forceinline__ dd dd_pi4() { return dd{7.853981633974483096e-01, 3.061616997868383e-17}; }

// sin and cos of x in [0, pi/4] by their Taylor series (15 terms each: the next term
// is below 1e-34).
__device__ __forceinline__ void dd_sincos_small(dd x, dd& s, dd& c) {
  const dd x2 = dd_mul(x, x);
  dd ts = x, tc = dd{1.0, 0.0};
  s = x;
  c = tc;
  for (int k = 1; k <= 15; ++k) {
    ts = dd_neg(dd_div_d(dd_mul(ts, x2), (double)((2 * k) * (2 * k + 1))));
    tc = dd_neg(dd_div_d(dd_mul(tc, x2), (double)((2 * k - 1) * (2 * k))));
    s = dd_add(s, ts);
    c = dd_add(c, tc);
  }
}

// cos and sin of 2 pi num / den (0 <= num < den < 2^50): the octant o of the angle and
// the remainder come from integer arithmetic, so multiples of pi / 4 are exact.
__device__ __forceinline__ void dd_cis_frac(int64_t num, int64_t den, dd& c, dd& s) {
  const int64_t a = 8 * num;
  const int o = (int)(a / den);
  const int64_t rem = a - (int64_t)o * den;  // angle = o pi/4 + (pi/4) rem / den
  const int64_t r2 = (o & 1) ? den - rem : rem;  // odd octant: pi/2 minus the angle in its quadrant
  const dd x = dd_mul(dd_pi4(), dd_div_d(dd{(double)r2, 0.0}, (double)den));
  dd sx, cx;
  dd_sincos_small(x, sx, cx);
  dd cq = (o & 1) ? sx : cx, sq = (o & 1) ? cx : sx;  // cos, sin of the angle within its quadrant
  switch ((o >> 1) & 3) {  // rotate by the quadrant
    case 0: c = cq; s = sq; break;
    case 1: c = dd_neg(sq); s = cq; break;
    case 2: c = dd_neg(cq); s = dd_neg(sq); break;
    default: c = sq; s = dd_neg(cq); break;
  }
}

// (cos, sin) as double-double from a table entry (cos hi, cos lo, sin hi, sin lo).
__device__ __forceinline__ void dd_from4(const double4& e, dd& c, dd& s) {
  c = dd{e.x, e.y};
  s = dd{e.z, e.w};
}

// omega = atan2(S, C) in double-double, S >= 0 and S^2 + C^2 = 1 (up to ~1e-32); anch:
// (cos, sin) of the anchors theta_j = j pi / 1024, j <= 1024, or null to compute them.
__device__ __forceinline__ dd dd_omega(dd S, dd C, const double4* __restrict__ anch) {
  const double w0 = atan2(S.hi, C.hi);
  int j = (int)rint(w0 * (1024.0 / 3.141592653589793116));
  j = j < 0 ? 0 : (j > 1024 ? 1024 : j);
  dd cj, sj;
  if (anch) dd_from4(anch[j], cj, sj);
  else dd_cis_frac(j, 2048, cj, sj);  // theta_j = 2 pi j / 2048
  const dd x = dd_sub(dd_mul(S, cj), dd_mul(C, sj));  // sin(omega - theta_j)
  // asin x = x + x^3/6 + 3x^5/40 + 5x^7/112 + 35x^9/1152 + ...  (|x| < 1.6e-3)
  const dd x3 = dd_mul(dd_mul(x, x), x);
  const double y = x.hi, y2 = y * y, y5 = y2 * y2 * y;
  const double tail = y5 * (0.075 + y2 * (5.0 / 112.0 + y2 * (35.0 / 1152.0)));
  dd w = dd_add(x, dd_div_d(x3, 6.0));
  w = dd_add(w, dd{tail, 0.0});
  const dd theta = dd_mul_d(dd_pi(), (double)j * (1.0 / 1024.0));
  return dd_add(theta, w);
}

}  // namespace qw
