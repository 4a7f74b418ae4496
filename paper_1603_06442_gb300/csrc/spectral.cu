// Fourier form of the walk (Sec. 4): psi(t) = IDFT[ D_k^t DFT[psi(0)] ].
//
// D_k^t in closed form.  With D_k = n u_k I - i G_k (Sec. 3.2; the Dirac block
// form gives G_k = [[n sigma.n~_k, -m I], [-m I, -n sigma.n~_k]], and in 1D
// G_k = [[n sin k, -m], [-m, -n sin k]]), G_k is Hermitian with
// G_k^2 = (m^2 + n^2 |n~_k|^2) I = sin^2(omega_k) I because u^2 + |n~|^2 = 1,
// so D_k = exp(-i omega_k G^_k) with G^_k = G_k / sin(omega_k) and
//     D_k^t = cos(omega_k t) I - i sin(omega_k t) G^_k ,
// the Chebyshev form (sin(omega t)/sin(omega) = U_{t-1}(cos omega)).
// omega_k = atan2(sin omega_k, n u_k) (the paper's arccos(n u_k), Sec. 3.2) is
// tabulated once per plan (BCC: for q0 only, see below): complex128 plans hold it as a
// double-double (~1e-31,
// qw_dd.cuh), so the phase omega_k t reduced modulo 2 pi carries ~1e-16 of
// rounding at any t instead of t ulp(omega_k); complex64 plans hold nu = omega/2pi
// as an FP32 pair for an FP32 phase.  Where sin(omega_k) = 0 (m = 0 and
// n~_k = 0) D_k = +-I and G^_k is taken as 0.
//
// BCC lattice (Eqs. bcc-dft, bcc-idft): the coset DFTs Psi^0, Psi^1 at the cell
// wave vector kappa in [0, 2 pi)^3 hold the two BCC wave vectors
// q0 = kappa/2 and q1 = kappa/2 + (pi, 0, 0); with a = exp(i (k1+k2+k3)/2),
//     c0 = (Psi^0 + a* Psi^1)/2,  c1 = (Psi^0 - a* Psi^1)/2,
// each evolves with its own D_q^t, and Psi^0 = c0 + c1, Psi^1 = a (c0 - c1).  q1 flips
// the signs of u and n~, so omega_q1 = pi - omega_q0 and D_q1^t = (-1)^t Gamma D_q0^t Gamma
// (Gamma = diag(I, -I)): the tables and G^ serve q0 alone.
// This is the paper's two-rectangular-DFT reduction written for the
// exp(-i k.x) forward convention.
#include <cuda_runtime.h>

#include <cmath>

#include "qw_dd.cuh"
#include "qw_spectral_dev.cuh"

namespace qw {

SpecAxes spec_axes(const Geometry& g, const FftPlan& f) {
  SpecAxes a;
  const int64_t ext[3] = {g.nx, g.ny, g.nz};
  for (int ax = 0; ax < 3; ++ax) {
    a.len[ax] = ext[ax];
    a.nparts[ax] = 1;
    a.part[ax][0] = (int)ext[ax];
    a.part[ax][1] = a.part[ax][2] = 1;
    if (ax < g.dim) {
      a.nparts[ax] = f.axis[ax].nparts;
      for (int q = 0; q < 3; ++q) a.part[ax][q] = q < f.axis[ax].nparts ? f.axis[ax].part[q] : 1;
    }
    a.trig[ax] = static_cast<const double2*>(f.trig[ax]);
    a.trig32[ax] = static_cast<const float2*>(f.trig32[ax]);
  }
  a.angle = static_cast<const double2*>(f.angle);
  for (int ax = 0; ax < 3; ++ax) a.trigdf[ax] = static_cast<const float4*>(f.trigdf[ax]);
  a.angdf = static_cast<const float4*>(f.angdf);
  return a;
}

// complex64 plans, per wave vector: nu = omega / (2 pi) (FP64) as an unevaluated FP32 pair
// (hi, lo), hi = RN(nu), lo = RN(nu - hi): |nu - hi - lo| <= 2^-48 nu, enough for the phase
// nu t of any t < 2^24 to ~1e-8 cycles with FP32 arithmetic.
__global__ void omega_split_kernel(int dim, AxesDev a, double n, double m, float2* __restrict__ nu_out) {
  int64_t x, y, z;
  if (grid_pos(a, x, y, z)) {
    const int64_t idx = (z * a.len[1] + y) * a.len[0] + x;
    int64_t f[3], fs;
    wave_vectors(dim, x, y, z, a, f, fs);
    double u, nx, ny, nz;
    symbol_tab<double>(dim, a, f[0], f[1], f[2], 0, u, nx, ny, nz);
    const double sw = sqrt(m * m + n * n * (nx * nx + ny * ny + nz * nz));
    const double nu = atan2(sw, n * u) * 0.15915494309189533577;
    const float hi = (float)nu;
    nu_out[idx] = make_float2(hi, (float)(nu - (double)hi));
  }
}

// (cos, sin)(2 pi q / period) for q < len as double-double (cos hi, cos lo, sin hi, sin lo).
__global__ void dd_table_kernel(double4* __restrict__ out, int64_t len, int64_t period) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= len) return;
  dd c, s;
  dd_cis_frac(q % period, period, c, s);
  out[q] = make_double4(c.hi, c.lo, s.hi, s.lo);
}

// n = sqrt(1 - m^2) as double-double (m is exact in FP64)
__global__ void dd_mass_kernel(double m, double2* out) {
  const dd n = dd_sqrt(dd_sub(dd{1.0, 0.0}, dd_two_prod(m, m)));
  *out = make_double2(n.hi, n.lo);
}

// complex128 plans: omega_k as a double-double (hi, lo) per stored wave vector, from the
// symbol in double-double: per-axis tables of the same angles as the FP64 tables (2D:
// pi q / N, q < 2N; BCC: the half angles pi f / M; the chain's 2 pi f / N is computed
// directly) and the anchors of dd_omega.
__global__ void omega_dd_kernel(int dim, AxesDev a, double m, const double2* __restrict__ nbox,
                                const double4* __restrict__ tab0, const double4* __restrict__ tab1,
                                const double4* __restrict__ tab2, const double4* __restrict__ anch,
                                double2* __restrict__ omega) {
  int64_t x, y, z;
  if (!grid_pos(a, x, y, z)) return;
  const int64_t idx = (z * a.len[1] + y) * a.len[0] + x;
  int64_t f[3], fs;
  wave_vectors(dim, x, y, z, a, f, fs);
  const dd n = dd{nbox->x, nbox->y};
  const dd m2 = dd_two_prod(m, m), n2 = dd_mul(n, n);
  {
    dd u, t1, t2, t3;  // u_k and n~_k (Eqs. weyl1d, weyl2d, weyl3d)
    if (dim == 1) {
      dd c, s;
      dd_cis_frac(f[0], a.len[0], c, s);
      u = c;
      t1 = dd{0.0, 0.0};
      t2 = t1;
      t3 = s;
    } else if (dim == 2) {
      const int64_t N2 = 2 * a.len[0];
      int64_t dm = f[0] - f[1];
      if (dm < 0) dm += N2;
      dd cx, sx, cy, sy;
      dd_from4(tab0[f[0] + f[1]], cx, sx);
      dd_from4(tab0[dm], cy, sy);
      u = dd_mul(cx, cy);
      t1 = dd_mul(sx, cy);
      t2 = dd_mul(cx, sy);
      t3 = dd_mul(sx, sy);
    } else {
      dd cx, sx, cy, sy, cz, sz;
      dd_from4(tab0[f[0]], cx, sx);
      dd_from4(tab1[f[1]], cy, sy);
      dd_from4(tab2[f[2]], cz, sz);
      u = dd_add(dd_mul(dd_mul(cx, cy), cz), dd_mul(dd_mul(sx, sy), sz));
      t1 = dd_sub(dd_mul(dd_mul(sx, cy), cz), dd_mul(dd_mul(cx, sy), sz));
      t2 = dd_add(dd_mul(dd_mul(cx, sy), cz), dd_mul(dd_mul(sx, cy), sz));
      t3 = dd_sub(dd_mul(dd_mul(cx, cy), sz), dd_mul(dd_mul(sx, sy), cz));
    }
    const dd nt2 = dd_add(dd_add(dd_mul(t1, t1), dd_mul(t2, t2)), dd_mul(t3, t3));
    const dd S = dd_sqrt(dd_add(m2, dd_mul(n2, nt2)));  // sin omega
    const dd w = dd_omega(S, dd_mul(n, u), anch);
    omega[idx] = make_double2(w.hi, w.lo);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) evolve_kernel(int dim, AxesDev a, int64_t count, Mass ms,
                                                     const double* __restrict__ omega, TimeArg ta, T scale_in,
                                                     const double* __restrict__ norm0,
                                                     typename Cx2<T>::t* __restrict__ data) {
  using V = typename Cx2<T>::t;
  // optional normalisation of the initial state, folded into the 1/|V| scale
  const T scale = norm0 ? (sizeof(T) == 8 ? (T)((double)scale_in / sqrt(norm0[0]))
                                           : (T)(scale_in * rsqrtf((float)norm0[0])))
                        : scale_in;
  int64_t x, y, z;
  if (grid_pos(a, x, y, z)) {
    const int64_t idx = (z * a.len[1] + y) * a.len[0] + x;
    const int P = planes_of(dim);
    V v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < P) v[q] = data[q * count + idx];
    evolve_point<T>(dim, a, x, y, z, idx, ms, omega, ta, scale, v);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < P) data[q * count + idx] = v[q];
  }
}

// Foldy-Wouthuysen coefficients of one wave vector (the Remark on the Newton-Wigner
// position): w_r = u_r(k)^dag v on the paper's eigenvectors of D_k (Eq. evecs-D),
// r = (s, p) in the order (+,+), (+,-), (-,+), (-,-):
//   u_{s,p} = (A, -p B e^{i phi}, -s C, s p D) / 2,  A = sqrt((1 - p vW)(1 + s p vD)),
//   B = sqrt((1 + p vW)(1 + s p vD)), C = sqrt((1 - p vW)(1 - s p vD)), D = sqrt((1 + p vW)(1 - s p vD)),
// vW = -n~_z / |n~|, e^{i phi} = -(n~_x + i n~_y) / |(n~_x, n~_y)| (phi = Arg(n~_y - i n~_x) - pi/2),
// vD = n |n~| / sqrt(m^2 + n^2 |n~|^2); vW = 0, phi = 0, vD = 0 where their ratios are 0/0.
// 1D (the decoupled 2x2 walk): u_+ = (cos th/2, -sin th/2), u_- = (sin th/2, cos th/2),
// th = atan2(m, n sin k).
template <typename T, int S>
__device__ __forceinline__ void fw_apply(T u, T nx, T ny, T nz, T n, T m, typename Cx2<T>::t (&v)[S]) {
  using V = typename Cx2<T>::t;
  (void)u;
  if (S == 2) {
    const T th = atan2(m, n * nz);
    const T c = cos((T)0.5 * th), sn = sin((T)0.5 * th);
    const V a = v[0], b = v[1];
    v[0].x = c * a.x - sn * b.x;
    v[0].y = c * a.y - sn * b.y;
    v[1].x = sn * a.x + c * b.x;
    v[1].y = sn * a.y + c * b.y;
    return;
  }
  const T tiny = sizeof(T) == 8 ? (T)1e-12 : (T)1e-6;
  const T r = sqrt(nx * nx + ny * ny + nz * nz);
  T vW = r < tiny ? (T)0 : -nz / r;
  vW = vW > (T)1 ? (T)1 : (vW < (T)-1 ? (T)-1 : vW);
  const T wa = sqrt(nx * nx + ny * ny);
  const T ec = wa > tiny ? -nx / wa : (T)1, es = wa > tiny ? -ny / wa : (T)0;
  const T den = sqrt(m * m + n * n * r * r);
  T vD = den > tiny ? n * r / den : (T)0;
  vD = vD > (T)1 ? (T)1 : (vD < (T)-1 ? (T)-1 : vD);
  // e^{-i phi} v1, e^{-i phi} v3
  V t1, t3;
  t1.x = ec * v[1].x + es * v[1].y;
  t1.y = ec * v[1].y - es * v[1].x;
  t3.x = ec * v[3].x + es * v[3].y;
  t3.y = ec * v[3].y - es * v[3].x;
  V w[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const T sg = q < 2 ? (T)1 : (T)-1, pp = (q & 1) ? (T)-1 : (T)1;
    const T A = (T)0.5 * sqrt(((T)1 - pp * vW) * ((T)1 + sg * pp * vD));
    const T B = (T)0.5 * sqrt(((T)1 + pp * vW) * ((T)1 + sg * pp * vD));
    const T C = (T)0.5 * sqrt(((T)1 - pp * vW) * ((T)1 - sg * pp * vD));
    const T D = (T)0.5 * sqrt(((T)1 + pp * vW) * ((T)1 - sg * pp * vD));
    w[q].x = A * v[0].x - pp * B * t1.x - sg * C * v[2].x + sg * pp * D * t3.x;
    w[q].y = A * v[0].y - pp * B * t1.y - sg * C * v[2].y + sg * pp * D * t3.y;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = w[q];
}

template <typename T>
__global__ void __launch_bounds__(256) fw_kernel(int dim, AxesDev a, int64_t count, Mass ms, T scale,
                                                 typename Cx2<T>::t* __restrict__ data) {
  using V = typename Cx2<T>::t;
  int64_t x, y, z;
  if (!grid_pos(a, x, y, z)) return;
  const int64_t idx = (z * a.len[1] + y) * a.len[0] + x;
  const int P = planes_of(dim);
  const T n = sizeof(T) == 8 ? (T)ms.n : (T)ms.nf, m = sizeof(T) == 8 ? (T)ms.m : (T)ms.mf;
  V v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q)
    if (q < P) v[q] = data[q * count + idx];
  int64_t f[3], fs;
  wave_vectors(dim, x, y, z, a, f, fs);
  if (dim == 1) {
    V w[2] = {v[0], v[1]};
    T u, nx, ny, nz;
    symbol_tab<T>(1, a, f[0], f[1], f[2], 0, u, nx, ny, nz);
    fw_apply<T, 2>(u, nx, ny, nz, n, m, w);
    v[0] = make_vec(w[0], scale);
    v[1] = make_vec(w[1], scale);
  } else if (dim == 2) {
    V w[4] = {v[0], v[1], v[2], v[3]};
    T u, nx, ny, nz;
    symbol_tab<T>(2, a, f[0], f[1], f[2], 0, u, nx, ny, nz);
    fw_apply<T, 4>(u, nx, ny, nz, n, m, w);
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = make_vec(w[q], scale);
  } else {
    // BCC: the two wave vectors q0, q1 of the cell from the coset mix, as in evolve_point
    T ar, ai;
    coset_phase<T>(fs, a.len[0], ar, ai);
    V c0[4], c1[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      V b;
      b.x = ar * v[4 + q].x + ai * v[4 + q].y;
      b.y = ar * v[4 + q].y - ai * v[4 + q].x;
      c0[q].x = (T)0.5 * (v[q].x + b.x);
      c0[q].y = (T)0.5 * (v[q].y + b.y);
      c1[q].x = (T)0.5 * (v[q].x - b.x);
      c1[q].y = (T)0.5 * (v[q].y - b.y);
    }
    T u, nx, ny, nz;
    symbol_tab<T>(3, a, f[0], f[1], f[2], 0, u, nx, ny, nz);
    fw_apply<T, 4>(u, nx, ny, nz, n, m, c0);
    symbol_tab<T>(3, a, f[0], f[1], f[2], 1, u, nx, ny, nz);
    fw_apply<T, 4>(u, nx, ny, nz, n, m, c1);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      V s0, d, s1;
      s0.x = c0[q].x + c1[q].x;
      s0.y = c0[q].y + c1[q].y;
      d.x = c0[q].x - c1[q].x;
      d.y = c0[q].y - c1[q].y;
      s1.x = ar * d.x - ai * d.y;
      s1.y = ar * d.y + ai * d.x;
      v[q] = make_vec(s0, scale);
      v[4 + q] = make_vec(s1, scale);
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q)
    if (q < P) data[q * count + idx] = v[q];
}

// launch_fused<R1, R2> is instantiated in fused_x_*.cu
QW_FUSED_LENGTHS(QW_FUSED_X_EXTERN)

// Particle weight: sum |c|^2 and sum c^dag G^ c over every wave vector.
template <typename T>
__global__ void __launch_bounds__(256) weights_kernel(int dim, AxesDev a, int64_t count, Mass ms,
                                                      const typename Cx2<T>::t* __restrict__ data,
                                                      double* __restrict__ partials) {
  using V = typename Cx2<T>::t;
  double acc[2] = {0.0, 0.0};
  const int64_t nx = a.len[0], ny = a.len[1];
  const int P = planes_of(dim);
  // segments of up to 16 points summed in T, segment sums added in FP64
  T seg[2] = {(T)0, (T)0};
  int nseg = 0;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < count;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t x, y, z;
    if (count <= 0x7fffffff) {  // 32-bit index arithmetic for planes below 2^31 values
      const int i32 = (int)idx, nx32 = (int)nx, ny32 = (int)ny;
      const int yz = i32 / nx32;
      x = i32 - yz * nx32;
      y = yz % ny32;
      z = yz / ny32;
    } else {
      x = idx % nx;
      y = (idx / nx) % ny;
      z = idx / (nx * ny);
    }
    V v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < P) v[q] = data[q * count + idx];
    weights_point<T>(dim, a, x, y, z, ms, v, seg);
    if (++nseg == 16) {
      acc[0] += (double)seg[0];
      acc[1] += (double)seg[1];
      seg[0] = seg[1] = (T)0;
      nseg = 0;
    }
  }
  acc[0] += (double)seg[0];
  acc[1] += (double)seg[1];
  block_sum<2, 256>(acc);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = acc[0];
    partials[2 * blockIdx.x + 1] = acc[1];
  }
}

// Sum of nblk (a, b) partial pairs in a fixed order: 1024 threads, four independent
// accumulators per thread (the partial count reaches 10^5 for the x-pass weights).
constexpr int kFoldThreads = 1024;
__global__ void __launch_bounds__(kFoldThreads) fold2_kernel(const double* __restrict__ partials, int nblk,
                                                              double* __restrict__ result) {
  const double2* p = reinterpret_cast<const double2*>(partials);
  double a0[4] = {0.0, 0.0, 0.0, 0.0}, a1[4] = {0.0, 0.0, 0.0, 0.0};
  int b = threadIdx.x;
  for (; b + 3 * kFoldThreads < nblk; b += 4 * kFoldThreads) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const double2 v = p[b + u * kFoldThreads];
      a0[u] += v.x;
      a1[u] += v.y;
    }
  }
  for (; b < nblk; b += kFoldThreads) {
    const double2 v = p[b];
    a0[0] += v.x;
    a1[0] += v.y;
  }
  double acc[2] = {(a0[0] + a0[1]) + (a0[2] + a0[3]), (a1[0] + a1[1]) + (a1[2] + a1[3])};
  block_sum<2, kFoldThreads>(acc);
  if (threadIdx.x == 0) {
    result[0] = acc[0];
    result[1] = acc[1];
  }
}

static int64_t kcount(const Geometry& g) { return g.vol; }


static dim3 grid3(const Geometry& g) {
  return dim3((unsigned)((g.nx + 255) / 256), (unsigned)g.ny, (unsigned)g.nz);
}

// complex128 plans: the double-double omega table (16 bytes per stored wave vector).  The
// per-axis and anchor tables it needs live in one temporary buffer (synchronous).
static qw_status launch_omega_table_dd(const Geometry& g, const SpecAxes& ax, double m, double* omega,
                                       cudaStream_t st) {
  const int64_t ext[3] = {g.nx, g.ny, g.nz};
  int64_t len[3] = {0, 0, 0}, per[3] = {1, 1, 1};
  if (g.dim == 2) {
    len[0] = per[0] = 2 * g.nx;
  } else if (g.dim == 3) {
    for (int a = 0; a < 3; ++a) {
      len[a] = ext[a];
      per[a] = 2 * ext[a];
    }
  }
  int64_t total = 1025 + 1;  // the anchors, then n
  for (int a = 0; a < 3; ++a) total += len[a];
  double4* buf = nullptr;
  QW_CHECK_CUDA(cudaMalloc(&buf, total * sizeof(double4)));
  double4* anch = buf;
  double2* nbox = reinterpret_cast<double2*>(buf + 1025);
  const double4* tabs[3] = {nullptr, nullptr, nullptr};
  int64_t off = 1026;
  for (int a = 0; a < 3; ++a) {
    if (!len[a]) continue;
    dd_table_kernel<<<(unsigned)((len[a] + 255) / 256), 256, 0, st>>>(buf + off, len[a], per[a]);
    tabs[a] = buf + off;
    off += len[a];
  }
  dd_table_kernel<<<5, 256, 0, st>>>(anch, 1025, 2048);
  dd_mass_kernel<<<1, 1, 0, st>>>(m, nbox);
  omega_dd_kernel<<<grid3(g), 256, 0, st>>>(g.dim, to_dev(ax), m, nbox, tabs[0], tabs[1], tabs[2], anch,
                                            reinterpret_cast<double2*>(omega));
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "double-double omega table");
  return QW_OK;
}

qw_status launch_omega_table(const Geometry& g, const SpecAxes& ax, double n, double m, double* omega,
                              cudaStream_t st, bool split) {
  if (!split) return launch_omega_table_dd(g, ax, m, omega, st);
  omega_split_kernel<<<grid3(g), 256, 0, st>>>(g.dim, to_dev(ax), n, m, reinterpret_cast<float2*>(omega));
  QW_CHECK_LAUNCH("omega table launch");
  return QW_OK;
}

qw_status launch_evolve_pointwise(const Geometry& g, const SpecAxes& ax, qw_dtype dt, double n, double m,
                                  const double* omega, int64_t t, void* psi_hat, cudaStream_t st,
                                  const double* norm0) {
  const int64_t count = kcount(g);
  const double inv = 1.0 / (double)g.vol;
  if (dt == QW_C64)
    evolve_kernel<float><<<grid3(g), 256, 0, st>>>(g.dim, to_dev(ax), count, make_mass(n, m), omega,
                                                         make_time(t), (float)inv, norm0,
                                                         static_cast<float2*>(psi_hat));
  else
    evolve_kernel<double><<<grid3(g), 256, 0, st>>>(g.dim, to_dev(ax), count, make_mass(n, m), omega,
                                                          make_time(t), inv, norm0, static_cast<double2*>(psi_hat));
  QW_CHECK_LAUNCH("evolve launch");
  return QW_OK;
}

qw_status launch_fw_pointwise(const Geometry& g, const SpecAxes& ax, qw_dtype dt, double n, double m, void* psi_hat,
                              cudaStream_t st) {
  const int64_t count = kcount(g);
  const double inv = 1.0 / (double)g.vol;
  if (dt == QW_C64)
    fw_kernel<float><<<grid3(g), 256, 0, st>>>(g.dim, to_dev(ax), count, make_mass(n, m), (float)inv,
                                               static_cast<float2*>(psi_hat));
  else
    fw_kernel<double><<<grid3(g), 256, 0, st>>>(g.dim, to_dev(ax), count, make_mass(n, m), inv,
                                                static_cast<double2*>(psi_hat));
  QW_CHECK_LAUNCH("Foldy-Wouthuysen launch");
  return QW_OK;
}

bool fused_x_supported(const Geometry& g, const FftPlan& f, qw_dtype dt) {
  if (dt != QW_C64 || f.axis[0].count != 1 || g.dim < 2) return false;
  switch (g.nx) {
#define QW_FX(LEN, A, B) case LEN:
    QW_FUSED_LENGTHS(QW_FX)
#undef QW_FX
      return true;
    default:
      return false;
  }
}

qw_status launch_evolve_fused_x(const Geometry& g, const SpecAxes& ax, const FftPlan& f, double n, double m,
                                const double* omega, int64_t t, void* psi, cudaStream_t st, const double* norm0) {
  const void* tw = f.pass[f.axis[0].first].tw_line;
  switch (g.nx) {
#define QW_FX(LEN, A, B) \
  case LEN:              \
    return launch_fused<A, B>(g, ax, n, m, omega, t, psi, tw, st, norm0);
    QW_FUSED_LENGTHS(QW_FX)
#undef QW_FX
    default:
      set_error("fused x pass: no register kernel for length %lld", (long long)g.nx);
      return QW_EINVAL;
  }
}

int64_t fused_x_grid(const Geometry& g) {
  switch (g.nx) {
#define QW_FX(LEN, A, B) \
  case LEN:              \
    return fused_x_ctas<A, B>(g);
    QW_FUSED_LENGTHS(QW_FX)
#undef QW_FX
    default:
      return 0;
  }
}

qw_status launch_weights_fused_x(const Geometry& g, const SpecAxes& ax, const FftPlan& f, double n, double m,
                                 const void* data, double* partials, double* result, cudaStream_t st) {
  const void* tw = f.pass[f.axis[0].first].tw_line;
  qw_status s2 = QW_OK;
  switch (g.nx) {
#define QW_FX(LEN, A, B)                                                      \
  case LEN:                                                                   \
    s2 = launch_weights_x<A, B>(g, ax, n, m, data, tw, partials, st); \
    break;
    QW_FUSED_LENGTHS(QW_FX)
#undef QW_FX
    default:
      set_error("x-pass weights: no register kernel for length %lld", (long long)g.nx);
      return QW_EINVAL;
  }
  if (s2 != QW_OK) return s2;
  // partials holds 2 * (CTAs + kFoldCtas) doubles: the CTAs' pairs, then the fold's first stage
  const int64_t nblk = fused_x_grid(g);
  return launch_fold_partials(partials, nblk, 2, partials + 2 * nblk, result, st);
}

qw_status launch_particle_weights(const Geometry& g, const SpecAxes& ax, qw_dtype dt, double n, double m,
                                  const void* psi_hat, double* partials, double* result, cudaStream_t st) {
  const int64_t count = kcount(g);
  const int nblk = kObsBlocks;
  if (dt == QW_C64)
    weights_kernel<float><<<nblk, 256, 0, st>>>(g.dim, to_dev(ax), count, make_mass(n, m),
                                                static_cast<const float2*>(psi_hat), partials);
  else
    weights_kernel<double><<<nblk, 256, 0, st>>>(g.dim, to_dev(ax), count, make_mass(n, m),
                                                 static_cast<const double2*>(psi_hat), partials);
  QW_CHECK_LAUNCH("weights launch");
  fold2_kernel<<<1, kFoldThreads, 0, st>>>(partials, nblk, result);
  QW_CHECK_LAUNCH("fold launch");
  return QW_OK;
}

}  // namespace qw
