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

template <typename T>
__global__ void __launch_bounds__(256) packet_kernel(Geometry g, PacketArgs pa, typename CplxOf2<T>::t* psi) {
  using V = typename CplxOf2<T>::t;
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  const int64_t y = blockIdx.y, zc = blockIdx.z;
  const int c = g.dim == 3 ? (int)(zc & 1) : 0;
  const int64_t z = g.dim == 3 ? (zc >> 1) : 0;
  const double N = (double)g.N;
  const double scale = g.dim == 3 ? 2.0 : 1.0;
  const double pos[3] = {scale * (double)x + c, scale * (double)y + c, scale * (double)z + c};
  // displacements are exact in T (integers and half-integers below 2^24);
  // the envelope and phase are evaluated in the field's precision
  T r2 = 0, ph = 0;
  for (int j = 0; j < g.dim; ++j) {
    double d = pos[j] - pa.x0[j] + 0.5 * N;
    d = d - N * floor(d / N) - 0.5 * N;  // minimum image in [-N/2, N/2)
    const T dt = (T)d;
    r2 += dt * dt;
    ph += (T)pa.k0[j] * dt;
  }
  T sp, cp;
  if (sizeof(T) == 8) {
    double a, b;
    sincos((double)ph, &a, &b);
    sp = (T)a;
    cp = (T)b;
  } else {
    float a, b;
    sincosf((float)ph, &a, &b);
    sp = (T)a;
    cp = (T)b;
  }
  const T env = (sizeof(T) == 8) ? (T)exp(-(double)r2 * pa.inv4s2) : (T)expf(-(float)r2 * (float)pa.inv4s2);
  const int64_t cell = (z * g.ny + y) * g.nx + x;
  for (int q = 0; q < g.s; ++q) {
    const T cr = (T)pa.chi[2 * q], ci = (T)pa.chi[2 * q + 1];
    V v;
    v.x = env * (cp * cr - sp * ci);
    v.y = env * (cp * ci + sp * cr);
    psi[((int64_t)c * g.s + q) * g.vol + cell] = v;
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
  dim3 grid((unsigned)((g.nx + 255) / 256), (unsigned)g.ny, (unsigned)(g.nz * g.ncoset));
  if (dt == QW_C64)
    packet_kernel<float><<<grid, 256, 0, st>>>(g, pa, static_cast<float2*>(psi));
  else
    packet_kernel<double><<<grid, 256, 0, st>>>(g, pa, static_cast<double2*>(psi));
  QW_CHECK_LAUNCH("packet launch");
  return QW_OK;
}

}  // namespace qw
