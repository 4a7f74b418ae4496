// Synthetic initial states on the device: a Gaussian packet times a plane wave
// times a fixed spinor, the shape of the particle states of Sec. 5 (Definition 1,
// Figs. 2, 5, 6) written in position space.  The served path builds its
// inputs here so that no field crosses the host link.
#include <cuda_runtime.h>

#include "qw_internal.cuh"

namespace qw {

struct PacketArgs {
  double x0[3], k0[3], chi[8];
  double inv4s2;  // 1 / (4 sigma^2)
};

constexpr int kPacketRows = 8;  // y rows per CTA (2D and BCC): the x factor is reused across them

// One axis of the separable packet: exp(-d^2 / (4 sigma^2)) exp(i k0 d) at the
// lattice coordinate pos, d the minimum-image displacement from x0 in [-N/2, N/2).
// d and the phase k0 d (reduced modulo 2 pi) are formed in FP64, since d can
// exceed 2^24 on long chains; complex64 then takes expf / sincosf of the small
// reduced arguments, complex128 stays in FP64.
template <typename T>
__device__ __forceinline__ typename CplxOf2<T>::t axis_factor(double pos, double x0, double N, double invN, double k0,
                                                              double inv4s2) {
  double d = pos - x0 + 0.5 * N;
  d = fma(-N, floor(d * invN), d);
  d = d < 0.0 ? d + N : (d >= N ? d - N : d);  // guard the rounding of d * invN
  d -= 0.5 * N;
  const double arg = d * d * inv4s2;
  const double ph = k0 * d;
  const double r = fma(-6.283185307179586232, rint(ph * 0.15915494309189533577), ph);
  typename CplxOf2<T>::t v;
  if (sizeof(T) == 8) {
    double sn, cs;
    sincos(r, &sn, &cs);
    const double e = exp(-arg);
    v.x = (T)(e * cs);
    v.y = (T)(e * sn);
  } else {
    float sn, cs;
    sincosf((float)r, &sn, &cs);
    const float e = arg < 104.0 ? expf(-(float)arg) : 0.0f;
    v.x = (T)(e * cs);
    v.y = (T)(e * sn);
  }
  return v;
}

template <typename V>
__device__ __forceinline__ V cx_mul(V a, V b) {
  V r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

// grid (ceil(nx / 256), ceil(ny / kPacketRows), nz * ncoset); each CTA fills
// kPacketRows rows of one (z, coset) plane.
template <typename T>
__global__ void __launch_bounds__(256) packet_kernel(Geometry g, PacketArgs pa, typename CplxOf2<T>::t* psi) {
  using V = typename CplxOf2<T>::t;
  __shared__ V fyz[kPacketRows];
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t y0 = (int64_t)blockIdx.y * kPacketRows, zc = blockIdx.z;
  const int c = g.dim == 3 ? (int)(zc & 1) : 0;
  const int64_t z = g.dim == 3 ? (zc >> 1) : 0;
  const double N = (double)g.N, invN = 1.0 / N;
  const double scale = g.dim == 3 ? 2.0 : 1.0;
  const int rows = g.dim == 1 ? 1 : (int)((g.ny - y0) < kPacketRows ? (g.ny - y0) : kPacketRows);
  if (threadIdx.x < rows) {  // the y (and z) factors of this CTA's rows
    V f;
    f.x = (T)1;
    f.y = (T)0;
    if (g.dim >= 2)
      f = axis_factor<T>(scale * (double)(y0 + threadIdx.x) + c, pa.x0[1], N, invN, pa.k0[1], pa.inv4s2);
    if (g.dim == 3) f = cx_mul(f, axis_factor<T>(scale * (double)z + c, pa.x0[2], N, invN, pa.k0[2], pa.inv4s2));
    fyz[threadIdx.x] = f;
  }
  __syncthreads();
  if (x >= g.nx) return;
  const V fx = axis_factor<T>(scale * (double)x + c, pa.x0[0], N, invN, pa.k0[0], pa.inv4s2);
  V chi[4];
  for (int q = 0; q < g.s; ++q) {
    chi[q].x = (T)pa.chi[2 * q];
    chi[q].y = (T)pa.chi[2 * q + 1];
  }
  for (int r = 0; r < rows; ++r) {
    const V f = cx_mul(fx, fyz[r]);
    const int64_t cell = (z * g.ny + (y0 + r)) * g.nx + x;
    for (int q = 0; q < g.s; ++q) psi[((int64_t)c * g.s + q) * g.vol + cell] = cx_mul(f, chi[q]);
  }
}

qw_status launch_packet(const Geometry& g, qw_dtype dt, const double* x0, double sigma, const double* k0,
                        const double* chi, void* psi, cudaStream_t st) {
  if (!(sigma > 0.0)) {
    set_error("packet: sigma must be > 0");
    return QW_EINVAL;
  }
  PacketArgs pa;
  for (int j = 0; j < 3; ++j) {
    pa.x0[j] = x0[j];
    pa.k0[j] = k0[j];
  }
  for (int j = 0; j < 8; ++j) pa.chi[j] = chi[j];
  pa.inv4s2 = 1.0 / (4.0 * sigma * sigma);
  dim3 grid((unsigned)((g.nx + 255) / 256), (unsigned)((g.ny + kPacketRows - 1) / kPacketRows),
            (unsigned)(g.nz * g.ncoset));
  if (dt == QW_C64)
    packet_kernel<float><<<grid, 256, 0, st>>>(g, pa, static_cast<float2*>(psi));
  else
    packet_kernel<double><<<grid, 256, 0, st>>>(g, pa, static_cast<double2*>(psi));
  QW_CHECK_LAUNCH("packet launch");
  return QW_OK;
}

}  // namespace qw
