// Position-space observables (Sec. 5.2): the norm sum_x |psi(x)|^2 and the
// first moments sum_x x_i |psi(x)|^2 of the position operator X, in FP64.
//
// Each thread takes a segment of SEG consecutive x-cells of one row (fixed
// coset, z, y), sums the density and x*density over the segment in the field's
// precision, then adds the segment totals into FP64 accumulators (the y and z
// moments of a segment are y*norm and z*norm).  Warp-shuffle and shared-memory
// reductions give one partial per block; a single block then folds the
// partials in a fixed order, so the result is deterministic.
#include <cuda_runtime.h>

#include "qw_internal.cuh"

namespace qw {

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

__device__ __forceinline__ void block_sum4(double (&acc)[4]) { block_sum<4, kObsThreads>(acc); }

template <typename R, int SEG>
__global__ void __launch_bounds__(kObsThreads) moments_kernel(const typename Cplx<R>::T* __restrict__ psi,
                                                              Geometry g, double* __restrict__ partials) {
  using C = typename Cplx<R>::T;
  const int64_t segs_per_row = g.nx / SEG;
  const int64_t rows = (int64_t)g.ncoset * g.nz * g.ny;
  const int64_t nseg = rows * segs_per_row;
  const double scale = (g.dim == 3) ? 2.0 : 1.0;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t sidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; sidx < nseg;
       sidx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = sidx / segs_per_row;
    const int64_t x0 = (sidx - row * segs_per_row) * SEG;
    const int64_t y = row % g.ny;
    const int64_t zc = row / g.ny;
    const int64_t z = zc % g.nz;
    const int c = (int)(zc / g.nz);
    const C* base = psi + (int64_t)c * g.s * g.vol + (z * g.ny + y) * g.nx + x0;
    R nf = 0, xf = 0;
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
      R d = 0;
      for (int s = 0; s < g.s; ++s) {
        C v = __ldg(base + (int64_t)s * g.vol + j);
        d = fma(v.x, v.x, d);
        d = fma(v.y, v.y, d);
      }
      nf += d;
      xf = fma((R)j, d, xf);
    }
    const double n = (double)nf;
    const double off = (double)c;
    acc[0] += n;
    acc[1] += scale * ((double)xf + (double)x0 * n) + off * n;
    acc[2] += (scale * (double)y + off) * n;
    acc[3] += (scale * (double)z + off) * n;
  }
  block_sum4(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) partials[(int64_t)blockIdx.x * 4 + j] = acc[j];
  }
}

__global__ void __launch_bounds__(kObsThreads) fold_partials_kernel(const double* __restrict__ partials, int nblk,
                                                                    double* __restrict__ result) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] += partials[b * 4 + j];
  }
  block_sum4(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) result[j] = acc[j];
  }
}

// Second moments (the position covariance of Sec. 5.1's particle-state kinematics): per
// segment of SEG x-cells the density sums n = sum d, m1 = sum j d, m2 = sum j^2 d (j < SEG)
// in the field's precision, then, with X = X0 + sc j, Y and Z fixed on the segment, the ten
// FP64 sums  n, S_x, S_y, S_z, S_xx, S_yy, S_zz, S_xy, S_xz, S_yz.
constexpr int kMom2 = 10;
template <typename R, int SEG>
__global__ void __launch_bounds__(kObsThreads) moments2_kernel(const typename Cplx<R>::T* __restrict__ psi,
                                                               Geometry g, double* __restrict__ partials) {
  using C = typename Cplx<R>::T;
  const int64_t segs_per_row = g.nx / SEG;
  const int64_t rows = (int64_t)g.ncoset * g.nz * g.ny;
  const int64_t nseg = rows * segs_per_row;
  const double sc = (g.dim == 3) ? 2.0 : 1.0;
  double acc[kMom2];
#pragma unroll
  for (int j = 0; j < kMom2; ++j) acc[j] = 0.0;
  for (int64_t sidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; sidx < nseg;
       sidx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = sidx / segs_per_row;
    const int64_t x0 = (sidx - row * segs_per_row) * SEG;
    const int64_t y = row % g.ny;
    const int64_t zc = row / g.ny;
    const int64_t z = zc % g.nz;
    const int c = (int)(zc / g.nz);
    const C* base = psi + (int64_t)c * g.s * g.vol + (z * g.ny + y) * g.nx + x0;
    R nf = 0, m1 = 0, m2 = 0;
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
      R d = 0;
      for (int s = 0; s < g.s; ++s) {
        C v = __ldg(base + (int64_t)s * g.vol + j);
        d = fma(v.x, v.x, d);
        d = fma(v.y, v.y, d);
      }
      nf += d;
      m1 = fma((R)j, d, m1);
      m2 = fma((R)(j * j), d, m2);
    }
    const double n = (double)nf, M1 = (double)m1, M2 = (double)m2;
    const double off = (double)c;
    const double X0 = sc * (double)x0 + off;
    const double Y = g.dim >= 2 ? sc * (double)y + off : 0.0;
    const double Z = g.dim >= 3 ? sc * (double)z + off : 0.0;
    const double sx = fma(sc, M1, X0 * n);                       // sum X d
    const double sxx = fma(sc * sc, M2, X0 * fma(2.0 * sc, M1, X0 * n));  // sum X^2 d
    acc[0] += n;
    acc[1] += sx;
    acc[2] += Y * n;
    acc[3] += Z * n;
    acc[4] += sxx;
    acc[5] += Y * Y * n;
    acc[6] += Z * Z * n;
    acc[7] += Y * sx;
    acc[8] += Z * sx;
    acc[9] += Y * Z * n;
  }
  block_sum<kMom2, kObsThreads>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < kMom2; ++j) partials[(int64_t)blockIdx.x * kMom2 + j] = acc[j];
  }
}

__global__ void __launch_bounds__(kObsThreads) fold_moments2_kernel(const double* __restrict__ partials, int nblk,
                                                                    double* __restrict__ result) {
  double acc[kMom2];
#pragma unroll
  for (int j = 0; j < kMom2; ++j) acc[j] = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
#pragma unroll
    for (int j = 0; j < kMom2; ++j) acc[j] += partials[b * kMom2 + j];
  }
  block_sum<kMom2, kObsThreads>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < kMom2; ++j) result[j] = acc[j];
  }
}

template <typename R>
static void launch_moments2_t(const Geometry& g, const void* psi, double* partials, cudaStream_t st) {
  using C = typename Cplx<R>::T;
  const C* p = static_cast<const C*>(psi);
  if (g.nx % 16 == 0)
    moments2_kernel<R, 16><<<kObsBlocks, kObsThreads, 0, st>>>(p, g, partials);
  else if (g.nx % 4 == 0)
    moments2_kernel<R, 4><<<kObsBlocks, kObsThreads, 0, st>>>(p, g, partials);
  else
    moments2_kernel<R, 1><<<kObsBlocks, kObsThreads, 0, st>>>(p, g, partials);
}

qw_status launch_position_moments2(const Geometry& g, qw_dtype dt, const void* psi, double* partials,
                                   double* result, cudaStream_t st) {
  if (dt == QW_C64)
    launch_moments2_t<float>(g, psi, partials, st);
  else
    launch_moments2_t<double>(g, psi, partials, st);
  QW_CHECK_LAUNCH("second moments launch");
  fold_moments2_kernel<<<1, kObsThreads, 0, st>>>(partials, kObsBlocks, result);
  QW_CHECK_LAUNCH("second moments fold launch");
  return QW_OK;
}

template <typename R>
static void launch_moments_t(const Geometry& g, const void* psi, double* partials, cudaStream_t st) {
  using C = typename Cplx<R>::T;
  const C* p = static_cast<const C*>(psi);
  if (g.nx % 8 == 0)
    moments_kernel<R, 8><<<kObsBlocks, kObsThreads, 0, st>>>(p, g, partials);
  else if (g.nx % 4 == 0)
    moments_kernel<R, 4><<<kObsBlocks, kObsThreads, 0, st>>>(p, g, partials);
  else if (g.nx % 2 == 0)
    moments_kernel<R, 2><<<kObsBlocks, kObsThreads, 0, st>>>(p, g, partials);
  else
    moments_kernel<R, 1><<<kObsBlocks, kObsThreads, 0, st>>>(p, g, partials);
}

qw_status launch_position_moments(const Geometry& g, qw_dtype dt, const void* psi, double* partials,
                                  double* result, cudaStream_t st) {
  if (dt == QW_C64)
    launch_moments_t<float>(g, psi, partials, st);
  else
    launch_moments_t<double>(g, psi, partials, st);
  QW_CHECK_LAUNCH("moments launch");
  fold_partials_kernel<<<1, kObsThreads, 0, st>>>(partials, kObsBlocks, result);
  QW_CHECK_LAUNCH("fold launch");
  return QW_OK;
}

}  // namespace qw
