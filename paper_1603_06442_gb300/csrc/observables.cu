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

// Second moments (the position covariance of Sec. 5.1's particle-state kinematics): the
// ten FP64 sums n, S_x, S_y, S_z, S_xx, S_yy, S_zz, S_xy, S_xz, S_yz of the density over the
// position coordinates.  A thread owns one x column of one coset (X fixed) and a chunk of
// its (z, y) rows (the threads of a warp read consecutive x); it sums d, Y d, Z d, Y^2 d,
// Z^2 d, Y Z d over groups of four rows in the field's precision, then in FP64, and adds
// the X-weighted terms once per column.  One partial per block, folded in a fixed order.
constexpr int kMom2 = 10;
// S: spinor components (compile time, so that a group's loads are all issued before the sums)
template <typename R, int S>
__global__ void __launch_bounds__(kObsThreads) moments2_kernel(const typename Cplx<R>::T* __restrict__ psi,
                                                               Geometry g, int chunks, double* __restrict__ partials) {
  using C = typename Cplx<R>::T;
  const int64_t units = (int64_t)g.ncoset * g.nx;
  const int64_t rows = g.nz * g.ny;
  const int j = blockIdx.y;
  const int64_t r0 = j * rows / chunks, r1 = (j + 1) * rows / chunks;
  const int ny = (int)g.ny;
  const R sc = g.dim == 3 ? (R)2 : (R)1;
  double acc[kMom2];
#pragma unroll
  for (int q = 0; q < kMom2; ++q) acc[q] = 0.0;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < units;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(u / g.nx);
    const int64_t x = u - (int64_t)c * g.nx;
    const R off = g.dim == 3 ? (R)c : (R)0;
    const C* col = psi + (int64_t)c * g.s * g.vol + x;
    int z = (int)(r0 / ny), y = (int)(r0 - (int64_t)z * ny);
    double n = 0.0, sy = 0.0, sz = 0.0, syy = 0.0, szz = 0.0, syz = 0.0;
    for (int64_t r = r0; r < r1; r += 4) {
      // the group's (up to) four rows: every load first, then the sums
      C v[4][S];
      R Yk[4], Zk[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        Yk[k] = g.dim >= 2 ? sc * (R)y + off : (R)0;
        Zk[k] = g.dim >= 3 ? sc * (R)z + off : (R)0;
        if (r + k < r1) {
          const C* q = col + ((int64_t)z * ny + y) * g.nx;
#pragma unroll
          for (int s = 0; s < S; ++s) v[k][s] = q[(int64_t)s * g.vol];
        } else {
#pragma unroll
          for (int s = 0; s < S; ++s) v[k][s] = C{0, 0};
        }
        if (++y == ny) {
          y = 0;
          ++z;
        }
      }
      R gn = 0, gy = 0, gz = 0, gyy = 0, gzz = 0, gyz = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        R d = 0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
          d = fma(v[k][s].x, v[k][s].x, d);
          d = fma(v[k][s].y, v[k][s].y, d);
        }
        const R Y = Yk[k], Z = Zk[k];
        const R yd = Y * d, zd = Z * d;
        gn += d;
        gy += yd;
        gz += zd;
        gyy = fma(Y, yd, gyy);
        gzz = fma(Z, zd, gzz);
        gyz = fma(Y, zd, gyz);
      }
      n += (double)gn;
      sy += (double)gy;
      sz += (double)gz;
      syy += (double)gyy;
      szz += (double)gzz;
      syz += (double)gyz;
    }
    const double X = (double)(sc * (R)x + off);
    acc[0] += n;
    acc[1] += X * n;
    acc[2] += sy;
    acc[3] += sz;
    acc[4] += X * X * n;
    acc[5] += syy;
    acc[6] += szz;
    acc[7] += X * sy;
    acc[8] += X * sz;
    acc[9] += syz;
  }
  block_sum<kMom2, kObsThreads>(acc);
  if (threadIdx.x == 0) {
    const int64_t b = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
    for (int q = 0; q < kMom2; ++q) partials[b * kMom2 + q] = acc[q];
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
static int launch_moments2_t(const Geometry& g, const void* psi, double* partials, cudaStream_t st) {
  using C = typename Cplx<R>::T;
  const int64_t units = (int64_t)g.ncoset * g.nx, rows = g.nz * g.ny;
  int64_t bx = (units + kObsThreads - 1) / kObsThreads;
  if (bx > kMom2MaxBlocks / 2) bx = kMom2MaxBlocks / 2;
  // ~2^18 threads in all: chunks of the rows when the columns are few
  int64_t chunks = ((int64_t(1) << 18) + bx * kObsThreads - 1) / (bx * kObsThreads);
  if (chunks > rows) chunks = rows;
  if (chunks * bx > kMom2MaxBlocks) chunks = kMom2MaxBlocks / bx;
  if (chunks < 1) chunks = 1;
  if (g.s == 2)
    moments2_kernel<R, 2><<<dim3((unsigned)bx, (unsigned)chunks), kObsThreads, 0, st>>>(static_cast<const C*>(psi), g,
                                                                                        (int)chunks, partials);
  else
    moments2_kernel<R, 4><<<dim3((unsigned)bx, (unsigned)chunks), kObsThreads, 0, st>>>(static_cast<const C*>(psi), g,
                                                                                        (int)chunks, partials);
  return (int)(bx * chunks);
}

qw_status launch_position_moments2(const Geometry& g, qw_dtype dt, const void* psi, double* partials,
                                   double* result, cudaStream_t st) {
  const int nblk = (dt == QW_C64) ? launch_moments2_t<float>(g, psi, partials, st)
                                  : launch_moments2_t<double>(g, psi, partials, st);
  QW_CHECK_LAUNCH("second moments launch");
  fold_moments2_kernel<<<1, kObsThreads, 0, st>>>(partials, nblk, result);
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
