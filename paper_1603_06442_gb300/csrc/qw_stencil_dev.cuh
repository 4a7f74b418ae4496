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
// Each update has a core that takes pointers to component 0 of the cells it reads and a
// component stride, so that fields in global memory and tiles in shared memory (other
// pitches) run the same arithmetic in the same order.

// chain, s = 2: psi'_0(x) = n psi_0(x-1) + i m psi_1(x), psi'_1(x) = i m psi_0(x) + n psi_1(x+1)
template <bool NC, typename C, typename CF, typename I>
__device__ __forceinline__ void core_1d(const C* xm, const C* xp, const C* own, I cs, C* dst, I ds, const CF& cf) {
  C a = ldg<NC>(xm);        // psi_0(x - 1)
  C b = ldg<NC>(xp + cs);   // psi_1(x + 1)
  C o0 = ldg<NC>(own), o1 = ldg<NC>(own + cs);
  dst[0] = finish(cf, a, o1);
  dst[ds] = finish(cf, b, o0);
}

// (I: index type; the batched kernel's walks fit 32-bit indices)
template <typename R, bool NC = true, typename I = int64_t>
__device__ __forceinline__ void site_update_1d(const typename CplxOf<R>::T* __restrict__ in,
                                               typename CplxOf<R>::T* __restrict__ out, I N, I x,
                                               const typename CoefOf<R>::T& cf) {
  core_1d<NC>(in + wrapm<I>(x - 1, N), in + wrapm<I>(x + 1, N), in + x, N, out + x, N, cf);
}

// square lattice, s = 4 (tables above): the cells x-1, x+1, y-1, y+1 and the own cell
template <bool NC, typename C, typename CF, typename I>
__device__ __forceinline__ void core_2d(const C* sxm, const C* sxp, const C* sym, const C* syp, const C* own, I cs,
                                        C* dst, I ds, const CF& cf) {
  C S0 = {0, 0}, S1 = {0, 0}, S2 = {0, 0}, S3 = {0, 0};
  {  // h = +e1: source (x - 1, y)
    C a = ldg<NC>(sxm), b = ldg<NC>(sxm + cs), c = ldg<NC>(sxm + 2 * cs), d = ldg<NC>(sxm + 3 * cs);
    cmac<1, 1>(S0, a); cmac<1, -1>(S0, b); cmac<1, 1>(S1, a); cmac<1, -1>(S1, b);
    cmac<1, -1>(S2, c); cmac<-1, 1>(S2, d); cmac<-1, -1>(S3, c); cmac<1, 1>(S3, d);
  }
  {  // h = -e1: source (x + 1, y)
    C a = ldg<NC>(sxp), b = ldg<NC>(sxp + cs), c = ldg<NC>(sxp + 2 * cs), d = ldg<NC>(sxp + 3 * cs);
    cmac<1, 1>(S0, a); cmac<-1, 1>(S0, b); cmac<-1, -1>(S1, a); cmac<1, -1>(S1, b);
    cmac<1, -1>(S2, c); cmac<1, -1>(S2, d); cmac<1, 1>(S3, c); cmac<1, 1>(S3, d);
  }
  {  // h = +e2: source (x, y - 1)
    C a = ldg<NC>(sym), b = ldg<NC>(sym + cs), c = ldg<NC>(sym + 2 * cs), d = ldg<NC>(sym + 3 * cs);
    cmac<1, -1>(S0, a); cmac<1, 1>(S0, b); cmac<1, -1>(S1, a); cmac<1, 1>(S1, b);
    cmac<1, 1>(S2, c); cmac<-1, -1>(S2, d); cmac<-1, 1>(S3, c); cmac<1, -1>(S3, d);
  }
  {  // h = -e2: source (x, y + 1)
    C a = ldg<NC>(syp), b = ldg<NC>(syp + cs), c = ldg<NC>(syp + 2 * cs), d = ldg<NC>(syp + 3 * cs);
    cmac<1, -1>(S0, a); cmac<-1, -1>(S0, b); cmac<-1, 1>(S1, a); cmac<1, 1>(S1, b);
    cmac<1, 1>(S2, c); cmac<1, 1>(S2, d); cmac<1, -1>(S3, c); cmac<1, -1>(S3, d);
  }
  C o0 = ldg<NC>(own), o1 = ldg<NC>(own + cs), o2 = ldg<NC>(own + 2 * cs), o3 = ldg<NC>(own + 3 * cs);
  dst[0] = finish(cf, S0, o2);
  dst[ds] = finish(cf, S1, o3);
  dst[2 * ds] = finish(cf, S2, o0);
  dst[3 * ds] = finish(cf, S3, o1);
}

// site (x, y) of the N x N box
template <typename R, bool NC = true, typename I = int64_t>
__device__ __forceinline__ void site_update_2d(const typename CplxOf<R>::T* __restrict__ in,
                                               typename CplxOf<R>::T* __restrict__ out, I N, I x, I y,
                                               const typename CoefOf<R>::T& cf) {
  const I vol = N * N;
  const I xm = wrapm<I>(x - 1, N), xp = wrapm<I>(x + 1, N);
  const I ym = wrapm<I>(y - 1, N), yp = wrapm<I>(y + 1, N);
  const I i = y * N + x;
  core_2d<NC>(in + y * N + xm, in + y * N + xp, in + ym * N + x, in + yp * N + x, in + i, vol, out + i, vol, cf);
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

// src: component 0 of the other coset; (za, zb), (ya, yb), (xa, xb): its cells for h = +1 and
// h = -1 per axis, with pitches sz (z) and sy (y); own / dst: component 0 of the own cell.
template <bool NC, typename C, typename CF, typename I>
__device__ __forceinline__ void core_3d(const C* src, I sz, I sy, I za, I zb, I ya, I yb, I xa, I xb, I cs,
                                        const C* own, C* dst, I ds, const CF& cf) {
  C S0 = {0, 0}, S1 = {0, 0}, S2 = {0, 0}, S3 = {0, 0};
  bcc_term<+1, +1, +1, NC>(S0, S1, S2, S3, src + za * sz + ya * sy + xa, cs);
  bcc_term<+1, -1, +1, NC>(S0, S1, S2, S3, src + za * sz + yb * sy + xa, cs);
  bcc_term<-1, +1, +1, NC>(S0, S1, S2, S3, src + za * sz + ya * sy + xb, cs);
  bcc_term<-1, -1, +1, NC>(S0, S1, S2, S3, src + za * sz + yb * sy + xb, cs);
  bcc_term<+1, +1, -1, NC>(S0, S1, S2, S3, src + zb * sz + ya * sy + xa, cs);
  bcc_term<+1, -1, -1, NC>(S0, S1, S2, S3, src + zb * sz + yb * sy + xa, cs);
  bcc_term<-1, +1, -1, NC>(S0, S1, S2, S3, src + zb * sz + ya * sy + xb, cs);
  bcc_term<-1, -1, -1, NC>(S0, S1, S2, S3, src + zb * sz + yb * sy + xb, cs);
  C o0 = ldg<NC>(own), o1 = ldg<NC>(own + cs), o2 = ldg<NC>(own + 2 * cs), o3 = ldg<NC>(own + 3 * cs);
  dst[0] = finish(cf, S0, o2);
  dst[ds] = finish(cf, S1, o3);
  dst[2 * ds] = finish(cf, S2, o0);
  dst[3 * ds] = finish(cf, S3, o1);
}

template <typename R, bool NC = true, typename I = int64_t>
__device__ __forceinline__ void site_update_3d(const typename CplxOf<R>::T* __restrict__ in,
                                               typename CplxOf<R>::T* __restrict__ out, I M, int c, I z, I y, I x,
                                               const typename CoefOf<R>::T& cf) {
  const I plane = M * M, vol = plane * M;
  const I xa = wrapm<I>(x - 1 + c, M), xb = wrapm<I>(x + c, M);
  const I ya = wrapm<I>(y - 1 + c, M), yb = wrapm<I>(y + c, M);
  const I za = wrapm<I>(z - 1 + c, M), zb = wrapm<I>(z + c, M);
  const I i = z * plane + y * M + x;
  core_3d<NC>(in + (I)(1 - c) * 4 * vol, plane, M, za, zb, ya, yb, xa, xb, vol, in + (I)c * 4 * vol + i,
              out + (I)c * 4 * vol + i, vol, cf);
}

}  // namespace qw
