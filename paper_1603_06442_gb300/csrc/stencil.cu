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

namespace qw {

template <typename R> struct CplxOf;
template <> struct CplxOf<float> { using T = float2; };
template <> struct CplxOf<double> { using T = double2; };

template <typename C>
__device__ __forceinline__ C ldg(const C* p) { return __ldg(p); }

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

__device__ __forceinline__ int64_t wrapm(int64_t v, int64_t M) { return v < 0 ? v + M : (v >= M ? v - M : v); }

// ---------------------------------------------------------------- chain, s = 2
template <typename R>
__global__ void __launch_bounds__(256) step1d_kernel(const typename CplxOf<R>::T* __restrict__ in,
                                                     typename CplxOf<R>::T* __restrict__ out, int64_t N,
                                                     typename CoefOf<R>::T cf) {
  using C = typename CplxOf<R>::T;
  int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= N) return;
  const C* p0 = in;
  const C* p1 = in + N;
  C a = ldg(p0 + wrapm(x - 1, N));   // psi_0(x - 1)
  C b = ldg(p1 + wrapm(x + 1, N));   // psi_1(x + 1)
  C o0 = ldg(p0 + x), o1 = ldg(p1 + x);
  out[x] = finish(cf, a, o1);        // n psi_0(x-1) + i m psi_1(x)
  out[N + x] = finish(cf, b, o0);    // n psi_1(x+1) + i m psi_0(x)
}

// ------------------------------------------------------ square lattice, s = 4
template <typename R>
__global__ void __launch_bounds__(256) step2d_kernel(const typename CplxOf<R>::T* __restrict__ in,
                                                     typename CplxOf<R>::T* __restrict__ out, int64_t N,
                                                     typename CoefOf<R>::T cf) {
  using C = typename CplxOf<R>::T;
  int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t y = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= N || y >= N) return;
  const int64_t vol = N * N;
  const int64_t xm = wrapm(x - 1, N), xp = wrapm(x + 1, N);
  const int64_t ym = wrapm(y - 1, N), yp = wrapm(y + 1, N);
  C S0 = {0, 0}, S1 = {0, 0}, S2 = {0, 0}, S3 = {0, 0};
  {  // h = +e1: source (x - 1, y)
    const int64_t i = y * N + xm;
    C a = ldg(in + i), b = ldg(in + vol + i), c = ldg(in + 2 * vol + i), d = ldg(in + 3 * vol + i);
    cmac<1, 1>(S0, a); cmac<1, -1>(S0, b); cmac<1, 1>(S1, a); cmac<1, -1>(S1, b);
    cmac<1, -1>(S2, c); cmac<-1, 1>(S2, d); cmac<-1, -1>(S3, c); cmac<1, 1>(S3, d);
  }
  {  // h = -e1: source (x + 1, y)
    const int64_t i = y * N + xp;
    C a = ldg(in + i), b = ldg(in + vol + i), c = ldg(in + 2 * vol + i), d = ldg(in + 3 * vol + i);
    cmac<1, 1>(S0, a); cmac<-1, 1>(S0, b); cmac<-1, -1>(S1, a); cmac<1, -1>(S1, b);
    cmac<1, -1>(S2, c); cmac<1, -1>(S2, d); cmac<1, 1>(S3, c); cmac<1, 1>(S3, d);
  }
  {  // h = +e2: source (x, y - 1)
    const int64_t i = ym * N + x;
    C a = ldg(in + i), b = ldg(in + vol + i), c = ldg(in + 2 * vol + i), d = ldg(in + 3 * vol + i);
    cmac<1, -1>(S0, a); cmac<1, 1>(S0, b); cmac<1, -1>(S1, a); cmac<1, 1>(S1, b);
    cmac<1, 1>(S2, c); cmac<-1, -1>(S2, d); cmac<-1, 1>(S3, c); cmac<1, -1>(S3, d);
  }
  {  // h = -e2: source (x, y + 1)
    const int64_t i = yp * N + x;
    C a = ldg(in + i), b = ldg(in + vol + i), c = ldg(in + 2 * vol + i), d = ldg(in + 3 * vol + i);
    cmac<1, -1>(S0, a); cmac<-1, -1>(S0, b); cmac<-1, 1>(S1, a); cmac<1, 1>(S1, b);
    cmac<1, 1>(S2, c); cmac<1, 1>(S2, d); cmac<1, -1>(S3, c); cmac<1, -1>(S3, d);
  }
  const int64_t i = y * N + x;
  C o0 = ldg(in + i), o1 = ldg(in + vol + i), o2 = ldg(in + 2 * vol + i), o3 = ldg(in + 3 * vol + i);
  out[i] = finish(cf, S0, o2);
  out[vol + i] = finish(cf, S1, o3);
  out[2 * vol + i] = finish(cf, S2, o0);
  out[3 * vol + i] = finish(cf, S3, o1);
}

// ------------------------------------------------------------ BCC, s = 4
// Output coset c at cell m reads coset 1-c at (per axis) m - 1 + c for h = +1
// and m + c for h = -1: the site x - h of the other sublattice.
template <int HX, int HY, int HZ, typename C>
__device__ __forceinline__ void bcc_term(C& S0, C& S1, C& S2, C& S3, const C* __restrict__ src, int64_t vol) {
  constexpr int P = HX * HY * HZ;
  if constexpr (HZ == 1) {
    C a = ldg(src), b = ldg(src + vol), d = ldg(src + 3 * vol);
    cmac<1, -P>(S0, a);
    cmac<HX, -HY>(S0, b);
    cmac<-HX, HY>(S2, d);
    cmac<1, -P>(S3, d);
  } else {
    C a = ldg(src), b = ldg(src + vol), c = ldg(src + 2 * vol);
    cmac<HX, HY>(S1, a);
    cmac<1, -P>(S1, b);
    cmac<1, -P>(S2, c);
    cmac<-HX, -HY>(S3, c);
  }
}

template <typename R>
__global__ void __launch_bounds__(256) step3d_kernel(const typename CplxOf<R>::T* __restrict__ in,
                                                     typename CplxOf<R>::T* __restrict__ out, int64_t M,
                                                     typename CoefOf<R>::T cf) {
  using C = typename CplxOf<R>::T;
  int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t y = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
  int64_t zc = blockIdx.z;
  if (x >= M || y >= M) return;
  const int c = (int)(zc / M);
  const int64_t z = zc - (int64_t)c * M;
  const int64_t plane = M * M, vol = plane * M;
  // source coordinates: [h = +1] -> m - 1 + c, [h = -1] -> m + c
  const int64_t xa = wrapm(x - 1 + c, M), xb = wrapm(x + c, M);
  const int64_t ya = wrapm(y - 1 + c, M), yb = wrapm(y + c, M);
  const int64_t za = wrapm(z - 1 + c, M), zb = wrapm(z + c, M);
  const C* src = in + (int64_t)(1 - c) * 4 * vol;
  C S0 = {0, 0}, S1 = {0, 0}, S2 = {0, 0}, S3 = {0, 0};
  bcc_term<+1, +1, +1>(S0, S1, S2, S3, src + za * plane + ya * M + xa, vol);
  bcc_term<+1, -1, +1>(S0, S1, S2, S3, src + za * plane + yb * M + xa, vol);
  bcc_term<-1, +1, +1>(S0, S1, S2, S3, src + za * plane + ya * M + xb, vol);
  bcc_term<-1, -1, +1>(S0, S1, S2, S3, src + za * plane + yb * M + xb, vol);
  bcc_term<+1, +1, -1>(S0, S1, S2, S3, src + zb * plane + ya * M + xa, vol);
  bcc_term<+1, -1, -1>(S0, S1, S2, S3, src + zb * plane + yb * M + xa, vol);
  bcc_term<-1, +1, -1>(S0, S1, S2, S3, src + zb * plane + ya * M + xb, vol);
  bcc_term<-1, -1, -1>(S0, S1, S2, S3, src + zb * plane + yb * M + xb, vol);
  const int64_t i = z * plane + y * M + x;
  const C* own = in + (int64_t)c * 4 * vol + i;
  C o0 = ldg(own), o1 = ldg(own + vol), o2 = ldg(own + 2 * vol), o3 = ldg(own + 3 * vol);
  C* dst = out + (int64_t)c * 4 * vol + i;
  dst[0] = finish(cf, S0, o2);
  dst[vol] = finish(cf, S1, o3);
  dst[2 * vol] = finish(cf, S2, o0);
  dst[3 * vol] = finish(cf, S3, o1);
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
static qw_status launch_step_t(const Geometry& g, CF cf, const void* in, void* out, cudaStream_t st) {
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
    dim3 blk(32, 8), grd((unsigned)((g.nx + 31) / 32), (unsigned)((g.ny + 7) / 8), (unsigned)(2 * g.nz));
    step3d_kernel<R><<<grd, blk, 0, st>>>(src, dst, g.nx, cf);
  }
  QW_CHECK_LAUNCH("stencil step launch");
  return QW_OK;
}

qw_status launch_step(const Geometry& g, qw_dtype dt, double n, double m, const void* in, void* out,
                      cudaStream_t st) {
  if (dt == QW_C64) return launch_step_t<float>(g, make_coef32(g.dim, n, m), in, out, st);
  return launch_step_t<double>(g, make_coef64(g.dim, n, m), in, out, st);
}

}  // namespace qw
