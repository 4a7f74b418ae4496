// One step of the Dirac quantum walk in position space (Eq. upd-rule):
//     psi'(x) = U_0 psi(x) + sum_{h in S} U_h psi(x - h),
// with the transition matrices of the paper's symbols (Eqs. weyl1d/2d/3d and
// the Dirac coupling D_k = [[n W_k, i m], [i m, n W_k^dag]] of Sec. 3.2):
//   U_h = diag(n W_h, n W_{-h}^dag) for h != 0,  U_0 = [[0, i m I], [i m I, 0]].
//
// Derivation of W_h (update psi'(x) = sum_h W_h psi(x - h), symbol
// W_k = sum_h exp(-i k.h) W_h): with E_h = exp(-i k.h), cos k_j = (1/2) sum E and
// sin k_j = (i/2) sum h_j E, so every entry of W_h is (+-1 +- i)/4 or 0:
//   BCC (h in {+-1}^3, p = h_x h_y h_z):
//     h_z = +1: 4 W_h = [[1 - i p, h_x - i h_y], [0, 0]]
//     h_z = -1: 4 W_h = [[0, 0], [h_x + i h_y, 1 - i p]]
//   square lattice (k_x = (k1 + k2)/2, k_y = (k1 - k2)/2 in Eq. weyl2d):
//     4 W_{+e1} = [[1+i, 1-i], [1+i, 1-i]]     4 W_{-e1} = [[1+i, -1+i], [-1-i, 1-i]]
//     4 W_{+e2} = [[1-i, 1+i], [1-i, 1+i]]     4 W_{-e2} = [[1-i, -1-i], [-1+i, 1+i]]
//   chain: U_{+1} = [[n, 0], [0, 0]], U_{-1} = [[0, 0], [0, n]] (Sec. 3.2, 1D form).
// So every Weyl product is additions only; the factor n/4 and the mass term are
// applied once per output component (``finish``).
//
// These are the unfused kernels: one thread per lattice site (all components),
// neighbours read through the read-only path, one read + one write of the field
// per step in the ideal (64 B/site-step for s = 4 in complex64).
#include <cuda_runtime.h>

#include "qw_internal.cuh"
#include "qw_stencil_dev.cuh"

namespace qw {

// ---------------------------------------------------------------- plain kernels
template <typename R>
__global__ void __launch_bounds__(256) step1d_kernel(const typename CplxOf<R>::T* __restrict__ in,
                                                     typename CplxOf<R>::T* __restrict__ out, int64_t N,
                                                     typename CoefOf<R>::T cf) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < N) site_update_1d<R>(in, out, N, x, cf);
}

template <typename R>
__global__ void __launch_bounds__(256) step2d_kernel(const typename CplxOf<R>::T* __restrict__ in,
                                                     typename CplxOf<R>::T* __restrict__ out, int64_t N,
                                                     typename CoefOf<R>::T cf) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t y = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
  if (x < N && y < N) site_update_2d<R>(in, out, N, x, y, cf);
}

template <typename R>
__global__ void __launch_bounds__(256) step3d_kernel(const typename CplxOf<R>::T* __restrict__ in,
                                                     typename CplxOf<R>::T* __restrict__ out, int64_t M,
                                                     typename CoefOf<R>::T cf) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t y = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= M || y >= M) return;
  // blockIdx.z = 2 z + c: both cosets of a layer run together, so the layers
  // they share are still in L2 (a coset-major order reads the field twice).
  site_update_3d<R>(in, out, M, (int)(blockIdx.z & 1), (int64_t)(blockIdx.z >> 1), y, x, cf);
}

// ---------------------------------------------- BCC, s = 4, complex64, vectorised
// Each thread owns two neighbouring x-cells (one 16-byte float4 per component
// row).  The x-shifted neighbour a row needs (x0 - 1 for coset 0, x0 + 2 for
// coset 1) comes from the adjacent lane by shuffle; the lane at the warp edge
// loads it (with the periodic wrap).  Requires M % 64 == 0.
struct Row3 {
  float2 lo, mid, hi;  // source cells for [h_x = +1 of cell 0], [shared], [h_x = -1 of cell 1]
};

template <int C>
__device__ __forceinline__ Row3 load_row3(const float4* __restrict__ row, const float2* __restrict__ row2, int64_t xq,
                                          int64_t Mh, int lane) {
  const float4 v = __ldg(row + xq);
  Row3 r;
  if constexpr (C == 0) {
    // cell x0 needs x0 - 1 (h_x = +1) and x0 (h_x = -1); cell x0 + 1 needs x0, x0 + 1
    float lx = __shfl_up_sync(0xffffffffu, v.z, 1);
    float ly = __shfl_up_sync(0xffffffffu, v.w, 1);
    if (lane == 0) {
      const int64_t xl = (xq == 0) ? 2 * Mh - 1 : 2 * xq - 1;
      const float2 t = __ldg(row2 + xl);
      lx = t.x;
      ly = t.y;
    }
    r.lo = make_float2(lx, ly);
    r.mid = make_float2(v.x, v.y);
    r.hi = make_float2(v.z, v.w);
  } else {
    // cell x0 needs x0 (h_x = +1) and x0 + 1 (h_x = -1); cell x0 + 1 needs x0 + 1, x0 + 2
    float rx = __shfl_down_sync(0xffffffffu, v.x, 1);
    float ry = __shfl_down_sync(0xffffffffu, v.y, 1);
    if (lane == 31) {
      const int64_t xr = (xq == Mh - 1) ? 0 : 2 * xq + 2;
      const float2 t = __ldg(row2 + xr);
      rx = t.x;
      ry = t.y;
    }
    r.lo = make_float2(v.x, v.y);
    r.mid = make_float2(v.z, v.w);
    r.hi = make_float2(rx, ry);
  }
  return r;
}

// Accumulate the four h with the given (h_y, h_z) from the rows of one (y, z) source.
template <int HY, int HZ>
__device__ __forceinline__ void bcc_pair(float2 (&S)[2][4], const Row3& a, const Row3& b, const Row3& cd) {
  // h_x = +1: cell 0 reads lo, cell 1 reads mid;  h_x = -1: cell 0 reads mid, cell 1 reads hi
  constexpr int PP = 1 * HY * HZ, PM = -1 * HY * HZ;  // p for h_x = +1 / -1
  if constexpr (HZ == 1) {
    // S0 += (1 - i p) a + (h_x - i h_y) b ;  S2 += (-h_x + i h_y) d ;  S3 += (1 - i p) d
    cmac<1, -PP>(S[0][0], a.lo);  cmac<1, -HY>(S[0][0], b.lo);  cmac<-1, HY>(S[0][2], cd.lo);  cmac<1, -PP>(S[0][3], cd.lo);
    cmac<1, -PP>(S[1][0], a.mid); cmac<1, -HY>(S[1][0], b.mid); cmac<-1, HY>(S[1][2], cd.mid); cmac<1, -PP>(S[1][3], cd.mid);
    cmac<1, -PM>(S[0][0], a.mid); cmac<-1, -HY>(S[0][0], b.mid); cmac<1, HY>(S[0][2], cd.mid); cmac<1, -PM>(S[0][3], cd.mid);
    cmac<1, -PM>(S[1][0], a.hi);  cmac<-1, -HY>(S[1][0], b.hi);  cmac<1, HY>(S[1][2], cd.hi);  cmac<1, -PM>(S[1][3], cd.hi);
  } else {
    // S1 += (h_x + i h_y) a + (1 - i p) b ;  S2 += (1 - i p) c ;  S3 += (-h_x - i h_y) c
    cmac<1, HY>(S[0][1], a.lo);  cmac<1, -PP>(S[0][1], b.lo);  cmac<1, -PP>(S[0][2], cd.lo);  cmac<-1, -HY>(S[0][3], cd.lo);
    cmac<1, HY>(S[1][1], a.mid); cmac<1, -PP>(S[1][1], b.mid); cmac<1, -PP>(S[1][2], cd.mid); cmac<-1, -HY>(S[1][3], cd.mid);
    cmac<-1, HY>(S[0][1], a.mid); cmac<1, -PM>(S[0][1], b.mid); cmac<1, -PM>(S[0][2], cd.mid); cmac<1, -HY>(S[0][3], cd.mid);
    cmac<-1, HY>(S[1][1], a.hi);  cmac<1, -PM>(S[1][1], b.hi);  cmac<1, -PM>(S[1][2], cd.hi);  cmac<1, -HY>(S[1][3], cd.hi);
  }
}

template <int C>
__device__ __forceinline__ void bcc_vec_body(const float2* __restrict__ in, float2* __restrict__ out, int64_t M,
                                             const Coef32& cf, int64_t xq, int64_t y, int64_t z, int lane) {
  const int64_t plane = M * M, vol = plane * M, Mh = M / 2;
  const int64_t ya = wrapm(y - 1 + C, M), yb = wrapm(y + C, M);
  const int64_t za = wrapm(z - 1 + C, M), zb = wrapm(z + C, M);
  const float2* src = in + (int64_t)(1 - C) * 4 * vol;
  float2 S[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) S[j][q] = make_float2(0.f, 0.f);
  // h_z = +1 layer (za): components a, b, d
#pragma unroll
  for (int iy = 0; iy < 2; ++iy) {
    const int64_t ys = iy == 0 ? ya : yb;  // iy = 0 -> h_y = +1, iy = 1 -> h_y = -1
    const float2* r = src + za * plane + ys * M;
    Row3 a = load_row3<C>(reinterpret_cast<const float4*>(r), r, xq, Mh, lane);
    Row3 b = load_row3<C>(reinterpret_cast<const float4*>(r + vol), r + vol, xq, Mh, lane);
    Row3 d = load_row3<C>(reinterpret_cast<const float4*>(r + 3 * vol), r + 3 * vol, xq, Mh, lane);
    if (iy == 0) bcc_pair<+1, +1>(S, a, b, d); else bcc_pair<-1, +1>(S, a, b, d);
  }
  // h_z = -1 layer (zb): components a, b, c
#pragma unroll
  for (int iy = 0; iy < 2; ++iy) {
    const int64_t ys = iy == 0 ? ya : yb;
    const float2* r = src + zb * plane + ys * M;
    Row3 a = load_row3<C>(reinterpret_cast<const float4*>(r), r, xq, Mh, lane);
    Row3 b = load_row3<C>(reinterpret_cast<const float4*>(r + vol), r + vol, xq, Mh, lane);
    Row3 c = load_row3<C>(reinterpret_cast<const float4*>(r + 2 * vol), r + 2 * vol, xq, Mh, lane);
    if (iy == 0) bcc_pair<+1, -1>(S, a, b, c); else bcc_pair<-1, -1>(S, a, b, c);
  }
  const int64_t i = z * plane + y * M;
  const float4* own = reinterpret_cast<const float4*>(in + (int64_t)C * 4 * vol + i);
  float4* dst = reinterpret_cast<float4*>(out + (int64_t)C * 4 * vol + i);
  const int64_t v4 = vol / 2;
  float4 o[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) o[q] = __ldg(own + q * v4 + xq);
  // mass partner of component q: 0<->2, 1<->3
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 w = o[q ^ 2];
    const float2 r0 = finish(cf, S[0][q], make_float2(w.x, w.y));
    const float2 r1 = finish(cf, S[1][q], make_float2(w.z, w.w));
    dst[q * v4 + xq] = make_float4(r0.x, r0.y, r1.x, r1.y);
  }
}

__global__ void __launch_bounds__(256) step3d_c64_vec_kernel(const float2* __restrict__ in, float2* __restrict__ out,
                                                             int64_t M, Coef32 cf) {
  const int64_t xq = (int64_t)blockIdx.x * 32 + threadIdx.x;
  const int64_t y = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
  const int c = (int)(blockIdx.z & 1);
  const int64_t z = blockIdx.z >> 1;
  if (c == 0)
    bcc_vec_body<0>(in, out, M, cf, xq, y, z, threadIdx.x);
  else
    bcc_vec_body<1>(in, out, M, cf, xq, y, z, threadIdx.x);
}

Coef32 make_coef32(int dim, double n, double m) {
  const double nq = (dim == 1) ? n : 0.25 * n;
  Coef32 c;
  c.nq_hi = (float)nq;
  c.nq_lo = (float)(nq - (double)c.nq_hi);
  c.m_hi = (float)m;
  c.m_lo = (float)(m - (double)c.m_hi);
  return c;
}

Coef64 make_coef64(int dim, double n, double m) {
  Coef64 c;
  c.nq = (dim == 1) ? n : 0.25 * n;
  c.m = m;
  return c;
}

template <typename R, typename CF>
static qw_status launch_step_t(const Geometry& g, int variant, CF cf, const void* in, void* out, cudaStream_t st) {
  using C = typename CplxOf<R>::T;
  const C* src = static_cast<const C*>(in);
  C* dst = static_cast<C*>(out);
  if (g.dim == 1) {
    dim3 blk(256), grd((unsigned)((g.nx + 255) / 256));
    step1d_kernel<R><<<grd, blk, 0, st>>>(src, dst, g.nx, cf);
  } else if (g.dim == 2) {
    dim3 blk(32, 8), grd((unsigned)((g.nx + 31) / 32), (unsigned)((g.ny + 7) / 8));
    step2d_kernel<R><<<grd, blk, 0, st>>>(src, dst, g.nx, cf);
  } else {
    if constexpr (sizeof(R) == 4) {
      if (variant == QW_STENCIL_VEC && g.nx % 64 == 0) {
        dim3 blk(32, 8), grd((unsigned)(g.nx / 64), (unsigned)(g.ny / 8), (unsigned)(2 * g.nz));
        step3d_c64_vec_kernel<<<grd, blk, 0, st>>>(src, dst, g.nx, cf);
        QW_CHECK_LAUNCH("stencil step launch");
        return QW_OK;
      }
    }
    dim3 blk(32, 8), grd((unsigned)((g.nx + 31) / 32), (unsigned)((g.ny + 7) / 8), (unsigned)(2 * g.nz));
    step3d_kernel<R><<<grd, blk, 0, st>>>(src, dst, g.nx, cf);
  }
  QW_CHECK_LAUNCH("stencil step launch");
  return QW_OK;
}

bool stencil_supported(const Geometry& g, qw_dtype dt, int variant) {
  switch (variant) {
    case QW_STENCIL_PLAIN: return true;
    case QW_STENCIL_VEC: return g.dim == 3 && dt == QW_C64 && g.nx % 64 == 0;
    case QW_STENCIL_TMA: return dt == QW_C64 && tma_step_supported(g);  // item table built at plan creation
    case QW_STENCIL_TMA2: return dt == QW_C64 && tma2_step_supported(g);
    case QW_STENCIL_FUSED: {
      const int box[3] = {g.dim == 1 ? 2048 : 64, g.dim == 2 ? 16 : 8, 8};
      return fused_step_supported(g, dt, 2, box);
    }
    default: return false;
  }
}

qw_status launch_step(const Geometry& g, qw_dtype dt, int variant, double n, double m, const void* in, void* out,
                      cudaStream_t st) {
  if (dt == QW_C64) return launch_step_t<float>(g, variant, make_coef32(g.dim, n, m), in, out, st);
  return launch_step_t<double>(g, variant, make_coef64(g.dim, n, m), in, out, st);
}

}  // namespace qw
