// Per-site update of the Dirac walk shared by the plain and batched stencil
// kernels (derivation of the transition matrices at the top of stencil.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qw_internal.cuh"

namespace qw {

template <typename R> struct CplxOf;
template <> struct CplxOf<float> { using T = float2; };
template <> struct CplxOf<double> { using T = double2; };

// Loads of the field.  The read-only path (__ldg, ld.global.nc) is only valid
// while nothing in the same launch writes the field; the batched kernel, whose
// CTAs read what other CTAs wrote earlier in the launch, passes NC = false and
// uses ordinary loads, which the PTX memory model orders after the CTA's
// acquire (thread 0's ld.acquire.gpu, then bar.sync).
template <bool NC = true, typename C>
__device__ __forceinline__ C ldg(const C* p) {
  if constexpr (NC) return __ldg(p);
  else return *p;  // ordinary load: ordered after the CTA's acquire by the memory model
}

// acc += (A + i B) * v  for A, B in {-1, 0, 1}: additions only.
template <int A, int B, typename C>
__device__ __forceinline__ void cmac(C& acc, const C& v) {
  if constexpr (A == 1) { acc.x += v.x; acc.y += v.y; }
  if constexpr (A == -1) { acc.x -= v.x; acc.y -= v.y; }
  if constexpr (B == 1) { acc.x -= v.y; acc.y += v.x; }
  if constexpr (B == -1) { acc.x += v.y; acc.y -= v.x; }
}

// nq * S + i m * o  (FP32: hi/lo split coefficients through FMA chains).
__device__ __forceinline__ float2 finish(const Coef32& c, float2 S, float2 o) {
  float rx = -c.m_lo * o.y;
  rx = fmaf(c.nq_lo, S.x, rx);
  rx = fmaf(-c.m_hi, o.y, rx);
  rx = fmaf(c.nq_hi, S.x, rx);
  float ry = c.m_lo * o.x;
  ry = fmaf(c.nq_lo, S.y, ry);
  ry = fmaf(c.m_hi, o.x, ry);
  ry = fmaf(c.nq_hi, S.y, ry);
  return make_float2(rx, ry);
}
__device__ __forceinline__ double2 finish(const Coef64& c, double2 S, double2 o) {
  return make_double2(fma(c.nq, S.x, -c.m * o.y), fma(c.nq, S.y, c.m * o.x));
}

template <typename R> struct CoefOf;
template <> struct CoefOf<float> { using T = Coef32; };
template <> struct CoefOf<double> { using T = Coef64; };

template <typename I>
__device__ __forceinline__ I wrapm(I v, I M) { return v < 0 ? v + M : (v >= M ? v - M : v); }


// ------------------------------------------------------------ per-site updates
// chain, s = 2: psi'_0(x) = n psi_0(x-1) + i m psi_1(x), psi'_1(x) = i m psi_0(x) + n psi_1(x+1)
// (I: index type; the batched kernel's walks fit 32-bit indices)
template <typename R, bool NC = true, typename I = int64_t>
__device__ __forceinline__ void site_update_1d(const typename CplxOf<R>::T* __restrict__ in,
                                               typename CplxOf<R>::T* __restrict__ out, I N, I x,
                                               const typename CoefOf<R>::T& cf) {
  using C = typename CplxOf<R>::T;
  const C* p0 = in;
  const C* p1 = in + N;
  C a = ldg<NC>(p0 + wrapm<I>(x - 1, N));   // psi_0(x - 1)
  C b = ldg<NC>(p1 + wrapm<I>(x + 1, N));   // psi_1(x + 1)
  C o0 = ldg<NC>(p0 + x), o1 = ldg<NC>(p1 + x);
  out[x] = finish(cf, a, o1);
  out[N + x] = finish(cf, b, o0);
}

// square lattice, s = 4 (tables above), site (x, y) of the N x N box
template <typename R, bool NC = true, typename I = int64_t>
__device__ __forceinline__ void site_update_2d(const typename CplxOf<R>::T* __restrict__ in,
                                               typename CplxOf<R>::T* __restrict__ out, I N, I x, I y,
                                               const typename CoefOf<R>::T& cf) {
  using C = typename CplxOf<R>::T;
  const I vol = N * N;
  const I xm = wrapm<I>(x - 1, N), xp = wrapm<I>(x + 1, N);
  const I ym = wrapm<I>(y - 1, N), yp = wrapm<I>(y + 1, N);
  C S0 = {0, 0}, S1 = {0, 0}, S2 = {0, 0}, S3 = {0, 0};
  {  // h = +e1: source (x - 1, y)
    const I i = y * N + xm;
    C a = ldg<NC>(in + i), b = ldg<NC>(in + vol + i), c = ldg<NC>(in + 2 * vol + i), d = ldg<NC>(in + 3 * vol + i);
    cmac<1, 1>(S0, a); cmac<1, -1>(S0, b); cmac<1, 1>(S1, a); cmac<1, -1>(S1, b);
    cmac<1, -1>(S2, c); cmac<-1, 1>(S2, d); cmac<-1, -1>(S3, c); cmac<1, 1>(S3, d);
  }
  {  // h = -e1: source (x + 1, y)
    const I i = y * N + xp;
    C a = ldg<NC>(in + i), b = ldg<NC>(in + vol + i), c = ldg<NC>(in + 2 * vol + i), d = ldg<NC>(in + 3 * vol + i);
    cmac<1, 1>(S0, a); cmac<-1, 1>(S0, b); cmac<-1, -1>(S1, a); cmac<1, -1>(S1, b);
    cmac<1, -1>(S2, c); cmac<1, -1>(S2, d); cmac<1, 1>(S3, c); cmac<1, 1>(S3, d);
  }
  {  // h = +e2: source (x, y - 1)
    const I i = ym * N + x;
    C a = ldg<NC>(in + i), b = ldg<NC>(in + vol + i), c = ldg<NC>(in + 2 * vol + i), d = ldg<NC>(in + 3 * vol + i);
    cmac<1, -1>(S0, a); cmac<1, 1>(S0, b); cmac<1, -1>(S1, a); cmac<1, 1>(S1, b);
    cmac<1, 1>(S2, c); cmac<-1, -1>(S2, d); cmac<-1, 1>(S3, c); cmac<1, -1>(S3, d);
  }
  {  // h = -e2: source (x, y + 1)
    const I i = yp * N + x;
    C a = ldg<NC>(in + i), b = ldg<NC>(in + vol + i), c = ldg<NC>(in + 2 * vol + i), d = ldg<NC>(in + 3 * vol + i);
    cmac<1, -1>(S0, a); cmac<-1, -1>(S0, b); cmac<-1, 1>(S1, a); cmac<1, 1>(S1, b);
    cmac<1, 1>(S2, c); cmac<1, 1>(S2, d); cmac<1, -1>(S3, c); cmac<1, -1>(S3, d);
  }
  const I i = y * N + x;
  C o0 = ldg<NC>(in + i), o1 = ldg<NC>(in + vol + i), o2 = ldg<NC>(in + 2 * vol + i), o3 = ldg<NC>(in + 3 * vol + i);
  out[i] = finish(cf, S0, o2);
  out[vol + i] = finish(cf, S1, o3);
  out[2 * vol + i] = finish(cf, S2, o0);
  out[3 * vol + i] = finish(cf, S3, o1);
}

// BCC, s = 4: output coset c at cell (x, y, z) reads coset 1-c at (per axis)
// m - 1 + c for h = +1 and m + c for h = -1 (the site x - h of the other sublattice).
template <int HX, int HY, int HZ, bool NC = true, typename C, typename I>
__device__ __forceinline__ void bcc_term(C& S0, C& S1, C& S2, C& S3, const C* __restrict__ src, I vol) {
  constexpr int P = HX * HY * HZ;
  if constexpr (HZ == 1) {
    C a = ldg<NC>(src), b = ldg<NC>(src + vol), d = ldg<NC>(src + 3 * vol);
    cmac<1, -P>(S0, a);
    cmac<HX, -HY>(S0, b);
    cmac<-HX, HY>(S2, d);
    cmac<1, -P>(S3, d);
  } else {
    C a = ldg<NC>(src), b = ldg<NC>(src + vol), c = ldg<NC>(src + 2 * vol);
    cmac<HX, HY>(S1, a);
    cmac<1, -P>(S1, b);
    cmac<1, -P>(S2, c);
    cmac<-HX, -HY>(S3, c);
  }
}

template <typename R, bool NC = true, typename I = int64_t>
__device__ __forceinline__ void site_update_3d(const typename CplxOf<R>::T* __restrict__ in,
                                               typename CplxOf<R>::T* __restrict__ out, I M, int c, I z, I y, I x,
                                               const typename CoefOf<R>::T& cf) {
  using C = typename CplxOf<R>::T;
  const I plane = M * M, vol = plane * M;
  const I xa = wrapm<I>(x - 1 + c, M), xb = wrapm<I>(x + c, M);
  const I ya = wrapm<I>(y - 1 + c, M), yb = wrapm<I>(y + c, M);
  const I za = wrapm<I>(z - 1 + c, M), zb = wrapm<I>(z + c, M);
  const C* src = in + (I)(1 - c) * 4 * vol;
  C S0 = {0, 0}, S1 = {0, 0}, S2 = {0, 0}, S3 = {0, 0};
  bcc_term<+1, +1, +1, NC>(S0, S1, S2, S3, src + za * plane + ya * M + xa, vol);
  bcc_term<+1, -1, +1, NC>(S0, S1, S2, S3, src + za * plane + yb * M + xa, vol);
  bcc_term<-1, +1, +1, NC>(S0, S1, S2, S3, src + za * plane + ya * M + xb, vol);
  bcc_term<-1, -1, +1, NC>(S0, S1, S2, S3, src + za * plane + yb * M + xb, vol);
  bcc_term<+1, +1, -1, NC>(S0, S1, S2, S3, src + zb * plane + ya * M + xa, vol);
  bcc_term<+1, -1, -1, NC>(S0, S1, S2, S3, src + zb * plane + yb * M + xa, vol);
  bcc_term<-1, +1, -1, NC>(S0, S1, S2, S3, src + zb * plane + ya * M + xb, vol);
  bcc_term<-1, -1, -1, NC>(S0, S1, S2, S3, src + zb * plane + yb * M + xb, vol);
  const I i = z * plane + y * M + x;
  const C* own = in + (I)c * 4 * vol + i;
  C o0 = ldg<NC>(own), o1 = ldg<NC>(own + vol), o2 = ldg<NC>(own + 2 * vol), o3 = ldg<NC>(own + 3 * vol);
  C* dst = out + (I)c * 4 * vol + i;
  dst[0] = finish(cf, S0, o2);
  dst[vol] = finish(cf, S1, o3);
  dst[2 * vol] = finish(cf, S2, o0);
  dst[3 * vol] = finish(cf, S3, o1);
}

}  // namespace qw
