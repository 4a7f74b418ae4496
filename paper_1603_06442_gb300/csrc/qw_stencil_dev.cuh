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
__device__ __forceinline__ void core_1d(const C* xm, const C* xp, const C* own, I cs, C (&r)[2], const CF& cf) {
  C a = ldg<NC>(xm);        // psi_0(x - 1)
  C b = ldg<NC>(xp + cs);   // psi_1(x + 1)
  C o0 = ldg<NC>(own), o1 = ldg<NC>(own + cs);
  r[0] = finish(cf, a, o1);
  r[1] = finish(cf, b, o0);
}

// (I: index type; the batched kernel's walks fit 32-bit indices)
template <typename R, bool NC = true, typename I = int64_t>
__device__ __forceinline__ void site_update_1d(const typename CplxOf<R>::T* __restrict__ in,
                                               typename CplxOf<R>::T* __restrict__ out, I N, I x,
                                               const typename CoefOf<R>::T& cf) {
  typename CplxOf<R>::T r[2];
  core_1d<NC>(in + wrapm<I>(x - 1, N), in + wrapm<I>(x + 1, N), in + x, N, r, cf);
  out[x] = r[0];
  out[N + x] = r[1];
}

// Complex helpers of the factored updates: rho = 1 + i, rhob = 1 - i.
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C rho(C z) { return C{z.x - z.y, z.x + z.y}; }
template <typename C> __device__ __forceinline__ C rhob(C z) { return C{z.x + z.y, z.y - z.x}; }
template <typename C> __device__ __forceinline__ C addi(C a, C b) { return C{a.x - b.y, a.y + b.x}; }  // a + i b

// square lattice, s = 4: the four outputs from the cells A = x-1, B = x+1, C = y-1, D = y+1
// (sources of h = +e1, -e1, +e2, -e2) and the own cell.  From the tables above, rho = 1 + i:
//   S0 = (P + Q) + (U - V),  S1 = (P + Q) - (U - V),
//     P = rho A0 + rhob A1, Q = rhob C0 + rho C1, U = rho (B0 + i B1), V = rho (D1 + i D0);
//   S2 = rhob (a + b) + rho (c + d),  S3 = rho (b - a) + rhob (d - c),
//     a = A2 - A3, b = B2 + B3, c = C2 - C3, d = D2 + D3
// (56 real additions instead of 128 term by term), then the mass step (finish).
template <bool NC, typename C, typename CF, typename I>
__device__ __forceinline__ void core_2d(const C* sxm, const C* sxp, const C* sym, const C* syp, const C* own, I cs,
                                        C (&r)[4], const CF& cf) {
  const C A0 = ldg<NC>(sxm), A1 = ldg<NC>(sxm + cs), A2 = ldg<NC>(sxm + 2 * cs), A3 = ldg<NC>(sxm + 3 * cs);
  const C B0 = ldg<NC>(sxp), B1 = ldg<NC>(sxp + cs), B2 = ldg<NC>(sxp + 2 * cs), B3 = ldg<NC>(sxp + 3 * cs);
  const C C0 = ldg<NC>(sym), C1 = ldg<NC>(sym + cs), C2 = ldg<NC>(sym + 2 * cs), C3 = ldg<NC>(sym + 3 * cs);
  const C D0 = ldg<NC>(syp), D1 = ldg<NC>(syp + cs), D2 = ldg<NC>(syp + 2 * cs), D3 = ldg<NC>(syp + 3 * cs);
  const C P = addi(cadd(A0, A1), csub(A0, A1));  // rho A0 + rhob A1
  const C Q = addi(cadd(C0, C1), csub(C1, C0));  // rhob C0 + rho C1
  const C U = rho(addi(B0, B1));
  const C V = rho(addi(D1, D0));
  const C PQ = cadd(P, Q), UV = csub(U, V);
  const C S0 = cadd(PQ, UV), S1 = csub(PQ, UV);
  const C a = csub(A2, A3), b = cadd(B2, B3), c = csub(C2, C3), d = cadd(D2, D3);
  const C S2 = cadd(rhob(cadd(a, b)), rho(cadd(c, d)));
  const C S3 = cadd(rho(csub(b, a)), rhob(csub(d, c)));
  const C o0 = ldg<NC>(own), o1 = ldg<NC>(own + cs), o2 = ldg<NC>(own + 2 * cs), o3 = ldg<NC>(own + 3 * cs);
  r[0] = finish(cf, S0, o2);
  r[1] = finish(cf, S1, o3);
  r[2] = finish(cf, S2, o0);
  r[3] = finish(cf, S3, o1);
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
  typename CplxOf<R>::T r[4];
  core_2d<NC>(in + y * N + xm, in + y * N + xp, in + ym * N + x, in + yp * N + x, in + i, vol, r, cf);
#pragma unroll
  for (int q = 0; q < 4; ++q) out[i + q * vol] = r[q];
}

// BCC, s = 4: output coset c at cell (x, y, z) reads coset 1-c at (per axis) m - 1 + c for
// h = +1 and m + c for h = -1 (the site x - h of the other sublattice).  From the tables above,
// with the sources s_{hx hy} of the plane of h_z = +1 and t_{hx hy} of the plane of h_z = -1,
// components a, b, c, d, and rho = 1 + i:
//   S0 = rhob [(a_{++} + b_{++}) + (a_{--} - b_{--})] + rho [(a_{+-} + b_{+-}) + (a_{-+} - b_{-+})]   (s)
//   S1 = rho [(a_{++} + b_{++}) + (b_{--} - a_{--})] + rhob [(a_{+-} + b_{+-}) + (b_{-+} - a_{-+})]   (t)
//   S2 = rhob (d_{--} - d_{++}) + rho (d_{-+} - d_{+-})  (s)  +  rho (c_{++} + c_{--}) + rhob (c_{+-} + c_{-+})  (t)
//   S3 = rhob (d_{++} + d_{--}) + rho (d_{+-} + d_{-+})  (s)  +  rho (c_{--} - c_{++}) + rhob (c_{-+} - c_{+-})  (t)
// (88 real additions instead of 128 term by term), then the mass step (finish).
// src: component 0 of the other coset; (za, zb), (ya, yb), (xa, xb): its cells for h = +1 and
// h = -1 per axis, with pitches sz (z) and sy (y); own: component 0 of the own cell.
template <bool NC, typename C, typename CF, typename I>
__device__ __forceinline__ void core_3d(const C* src, I sz, I sy, I za, I zb, I ya, I yb, I xa, I xb, I cs,
                                        const C* own, C (&r)[4], const CF& cf) {
  C S0, S1, S2, S3;
  {  // h_z = +1: plane za, components a, b, d
    const C* pp = src + za * sz + ya * sy + xa;  // (h_x, h_y) = (+, +)
    const C* pm = src + za * sz + yb * sy + xa;  // (+, -)
    const C* mp = src + za * sz + ya * sy + xb;  // (-, +)
    const C* mm = src + za * sz + yb * sy + xb;  // (-, -)
    const C app = ldg<NC>(pp), bpp = ldg<NC>(pp + cs), dpp = ldg<NC>(pp + 3 * cs);
    const C apm = ldg<NC>(pm), bpm = ldg<NC>(pm + cs), dpm = ldg<NC>(pm + 3 * cs);
    const C amp = ldg<NC>(mp), bmp = ldg<NC>(mp + cs), dmp = ldg<NC>(mp + 3 * cs);
    const C amm = ldg<NC>(mm), bmm = ldg<NC>(mm + cs), dmm = ldg<NC>(mm + 3 * cs);
    S0 = cadd(rhob(cadd(cadd(app, bpp), csub(amm, bmm))), rho(cadd(cadd(apm, bpm), csub(amp, bmp))));
    S2 = cadd(rhob(csub(dmm, dpp)), rho(csub(dmp, dpm)));
    S3 = cadd(rhob(cadd(dpp, dmm)), rho(cadd(dpm, dmp)));
  }
  {  // h_z = -1: plane zb, components a, b, c
    const C* pp = src + zb * sz + ya * sy + xa;
    const C* pm = src + zb * sz + yb * sy + xa;
    const C* mp = src + zb * sz + ya * sy + xb;
    const C* mm = src + zb * sz + yb * sy + xb;
    const C app = ldg<NC>(pp), bpp = ldg<NC>(pp + cs), cpp = ldg<NC>(pp + 2 * cs);
    const C apm = ldg<NC>(pm), bpm = ldg<NC>(pm + cs), cpm = ldg<NC>(pm + 2 * cs);
    const C amp = ldg<NC>(mp), bmp = ldg<NC>(mp + cs), cmp = ldg<NC>(mp + 2 * cs);
    const C amm = ldg<NC>(mm), bmm = ldg<NC>(mm + cs), cmm = ldg<NC>(mm + 2 * cs);
    S1 = cadd(rho(cadd(cadd(app, bpp), csub(bmm, amm))), rhob(cadd(cadd(apm, bpm), csub(bmp, amp))));
    S2 = cadd(S2, cadd(rho(cadd(cpp, cmm)), rhob(cadd(cpm, cmp))));
    S3 = cadd(S3, cadd(rho(csub(cmm, cpp)), rhob(csub(cmp, cpm))));
  }
  const C o0 = ldg<NC>(own), o1 = ldg<NC>(own + cs), o2 = ldg<NC>(own + 2 * cs), o3 = ldg<NC>(own + 3 * cs);
  r[0] = finish(cf, S0, o2);
  r[1] = finish(cf, S1, o3);
  r[2] = finish(cf, S2, o0);
  r[3] = finish(cf, S3, o1);
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
  typename CplxOf<R>::T r[4];
  core_3d<NC>(in + (I)(1 - c) * 4 * vol, plane, M, za, zb, ya, yb, xa, xb, vol, in + (I)c * 4 * vol + i, r, cf);
  typename CplxOf<R>::T* dst = out + (I)c * 4 * vol + i;
#pragma unroll
  for (int q = 0; q < 4; ++q) dst[q * vol] = r[q];
}

}  // namespace qw
