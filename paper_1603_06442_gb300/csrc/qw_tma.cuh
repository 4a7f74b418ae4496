// TMA-staged BCC stencil helpers shared by the one-step and two-step kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "qw_internal.cuh"

namespace qw {
namespace zm {

constexpr int TX = 64;                    // tile width (cells); two x-cells per thread
constexpr int BXC = TX + 4;               // box cells along x: [x0 - 2, x0 + TX + 2)
constexpr int ROWF = 2 * BXC;             // floats per box row
constexpr long long kSpinLimit = 1ll << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false (and the error word set) if the copy never lands.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* err) {
  for (long long i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// acc += (A + i B) v for A, B in {-1, 0, 1}
template <int A, int B>
__device__ __forceinline__ void cmac(float2& acc, const float2& v) {
  if constexpr (A == 1) { acc.x += v.x; acc.y += v.y; }
  if constexpr (A == -1) { acc.x -= v.x; acc.y -= v.y; }
  if constexpr (B == 1) { acc.x -= v.y; acc.y += v.x; }
  if constexpr (B == -1) { acc.x += v.y; acc.y -= v.x; }
}

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

struct Row3 {
  float2 lo, mid, hi;
};

// Row of one component: cells [lo, mid, hi] = tile-local x q0-1+C .. q0+1+C (q0 = 2 tx).
template <int C>
__device__ __forceinline__ Row3 srow(const float* row, int tx) {
  Row3 r;
  if constexpr (C == 0) {  // box columns q0+1, q0+2, q0+3
    const float2 a = *reinterpret_cast<const float2*>(row + 4 * tx + 2);
    const float4 b = *reinterpret_cast<const float4*>(row + 4 * tx + 4);
    r.lo = a;
    r.mid = make_float2(b.x, b.y);
    r.hi = make_float2(b.z, b.w);
  } else {                 // box columns q0+2, q0+3, q0+4
    const float4 a = *reinterpret_cast<const float4*>(row + 4 * tx + 4);
    const float2 b = *reinterpret_cast<const float2*>(row + 4 * tx + 8);
    r.lo = make_float2(a.x, a.y);
    r.mid = make_float2(a.z, a.w);
    r.hi = b;
  }
  return r;
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// Neighbour sums S0..S3 of cell J (0: lo/mid, 1: mid/hi columns) from the source rows
// of the two z-layers (index 0: h_y = +1 row, 1: h_y = -1 row):
//   h_z = +1 layer: components a, b, d;  h_z = -1 layer: components a2, b2, c2.
// The transition matrices (entries (+-1 +- i)/4, derived in stencil.cu) give, per
// source layer, terms (1 - i p) v and (+-h_x +- i h_y) v with p = h_x h_y h_z;
// grouped over the four (h_x, h_y) neighbours of a layer, with v_{xy} the value at
// h = (x, y),
//   P = v_{++} + v_{--},  Q = v_{+-} + v_{-+},  U = v_{++} - v_{--},  V = v_{+-} - v_{-+},
// the sums of (1 -+ i h_x h_y) v are (P + Q) -+ i (P - Q) and those of (h_x -+ i h_y) v
// are (U + V) -+ i (U - V); 80 additions per cell instead of 128.
template <int J>
__device__ __forceinline__ float2 colp(const Row3& r) { return J == 0 ? r.lo : r.mid; }  // h_x = +1
template <int J>
__device__ __forceinline__ float2 colm(const Row3& r) { return J == 0 ? r.mid : r.hi; }  // h_x = -1

template <int J>
__device__ __forceinline__ void bcc_sums(float2 (&S)[4], const Row3 (&a)[2], const Row3 (&b)[2], const Row3 (&d)[2],
                                         const Row3 (&a2)[2], const Row3 (&b2)[2], const Row3 (&c2)[2]) {
  // h_z = +1
  const float2 PA = cadd(colp<J>(a[0]), colm<J>(a[1])), QA = cadd(colp<J>(a[1]), colm<J>(a[0]));
  const float2 UB = csub(colp<J>(b[0]), colm<J>(b[1])), VB = csub(colp<J>(b[1]), colm<J>(b[0]));
  const float2 PD = cadd(colp<J>(d[0]), colm<J>(d[1])), QD = cadd(colp<J>(d[1]), colm<J>(d[0]));
  const float2 UD = csub(colp<J>(d[0]), colm<J>(d[1])), VD = csub(colp<J>(d[1]), colm<J>(d[0]));
  // h_z = -1
  const float2 UA = csub(colp<J>(a2[0]), colm<J>(a2[1])), VA = csub(colp<J>(a2[1]), colm<J>(a2[0]));
  const float2 PB = cadd(colp<J>(b2[0]), colm<J>(b2[1])), QB = cadd(colp<J>(b2[1]), colm<J>(b2[0]));
  const float2 PC = cadd(colp<J>(c2[0]), colm<J>(c2[1])), QC = cadd(colp<J>(c2[1]), colm<J>(c2[0]));
  const float2 UC = csub(colp<J>(c2[0]), colm<J>(c2[1])), VC = csub(colp<J>(c2[1]), colm<J>(c2[0]));
  {  // S0 = sum (1 - i p) a + (h_x - i h_y) b   (h_z = +1)
    const float2 al = cadd(PA, UB), be = cadd(QA, VB), s = cadd(al, be), t = csub(al, be);
    S[0] = make_float2(s.x + t.y, s.y - t.x);
  }
  {  // S1 = sum (h_x + i h_y) a2 + (1 + i h_x h_y) b2   (h_z = -1)
    const float2 al = cadd(UA, PB), be = cadd(VA, QB), s = cadd(al, be), t = csub(al, be);
    S[1] = make_float2(s.x - t.y, s.y + t.x);
  }
  {  // S2 = sum (-h_x + i h_y) d + (1 + i h_x h_y) c2
    const float2 X = cadd(csub(PC, UD), csub(QC, VD)), Y = csub(cadd(PC, UD), cadd(QC, VD));
    S[2] = make_float2(X.x - Y.y, X.y + Y.x);
  }
  {  // S3 = sum (1 - i h_x h_y) d + (-h_x - i h_y) c2
    const float2 X = cadd(csub(PD, UC), csub(QD, VC)), Y = csub(cadd(PD, UC), cadd(QD, VC));
    S[3] = make_float2(X.x + Y.y, X.y - Y.x);
  }
}

// Outputs of coset C at layer z for the thread's two cells.
//   lay_a: other coset at the h_z = +1 source layer, lay_b: at the h_z = -1 layer
//   own:   coset C at layer z (mass term)
template <int C, int CS>
__device__ __forceinline__ void compute(const float* lay_a, const float* lay_b, const float* own, float4* dst,
                                        int64_t v4, const Coef32& cf, int tx, int ty) {
  // box row of the h_y = +1 source: ty + C, of h_y = -1: ty + 1 + C
  Row3 a[2], b[2], d[2], a2[2], b2[2], c2[2];
#pragma unroll
  for (int iy = 0; iy < 2; ++iy) {
    const float* base = lay_a + (ty + C + iy) * ROWF;
    a[iy] = srow<C>(base, tx);
    b[iy] = srow<C>(base + CS, tx);
    d[iy] = srow<C>(base + 3 * CS, tx);
    const float* bb = lay_b + (ty + C + iy) * ROWF;
    a2[iy] = srow<C>(bb, tx);
    b2[iy] = srow<C>(bb + CS, tx);
    c2[iy] = srow<C>(bb + 2 * CS, tx);
  }
  float2 S[2][4];
  bcc_sums<0>(S[0], a, b, d, a2, b2, c2);
  bcc_sums<1>(S[1], a, b, d, a2, b2, c2);
  const float* ob = own + (ty + 1) * ROWF + 4 * tx + 4;
  float4 o[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) o[q] = *reinterpret_cast<const float4*>(ob + q * CS);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 w = o[q ^ 2];
    const float2 r0 = finish(cf, S[0][q], make_float2(w.x, w.y));
    const float2 r1 = finish(cf, S[1][q], make_float2(w.z, w.w));
    dst[q * v4] = make_float4(r0.x, r0.y, r1.x, r1.y);
  }
}

// Periodic images of a tile's out-of-range box cells.  The region is the edge
// columns (all rows) plus the edge rows (remaining columns); the k-th cell of
// that list, k = tid + i * NTH, is thread tid's i-th fix-up.
template <int MAXF>
struct FixT {
  int n;
  int soff[MAXF];      // float offset inside a buffer
  int64_t goff[MAXF];  // complex offset inside one coset (comp * vol + y * M + x)
};

template <int TYv, int NTH, int MAXF>
__device__ __forceinline__ void fix_setup(FixT<MAXF>& fx, int x0, int y0, int M, int64_t vol, int tid, int* err) {
  constexpr int BYv = TYv + 2, CSv = BYv * ROWF;
  const bool xl = (x0 == 0), xr = (x0 + TX == M), yl = (y0 == 0), yr = (y0 + TYv == M);
  const int nxo = 2 * (int)xl + 2 * (int)xr, nyo = (int)yl + (int)yr;
  const int nA = BYv * nxo, nB = nyo * (BXC - nxo), per = nA + nB;
  const int total = 4 * per;
  if (total > MAXF * NTH) atomicExch(err, 2);  // cannot happen for the tile shapes used
  fx.n = 0;
#pragma unroll
  for (int i = 0; i < MAXF; ++i) {
    const int k = tid + i * NTH;
    fx.soff[i] = 0;
    fx.goff[i] = 0;
    if (k < total) {
      const int cp = k / per, j = k % per;
      int r, q;
      if (j < nA) {
        r = j / nxo;
        const int oc = j % nxo;
        q = (xl && oc < 2) ? oc : TX + 2 + (oc & 1);
      } else {
        const int jj = j - nA, w = BXC - nxo;
        r = (yl && jj / w == 0) ? 0 : BYv - 1;
        q = (jj % w) + (xl ? 2 : 0);
      }
      int x = x0 - 2 + q, y = y0 - 1 + r;
      x = x < 0 ? x + M : (x >= M ? x - M : x);
      y = y < 0 ? y + M : (y >= M ? y - M : y);
      fx.soff[i] = cp * CSv + r * ROWF + 2 * q;
      fx.goff[i] = (int64_t)cp * vol + (int64_t)y * M + x;
      fx.n = i + 1;
    }
  }
}

}  // namespace zm
}  // namespace qw
