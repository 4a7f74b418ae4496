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

#include <type_traits>

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
// position coordinates.
//
// The covariance is a small difference of large raw moments, so a coordinate product must
// not be rounded in the field's precision: its error would be scaled by the coordinate
// itself, not by the packet's width.  A thread owns a unit (W adjacent x of one coset, W = 2
// for complex64 with one 16-byte load per component) and a chunk of its storage rows, which
// it takes in groups of up to G rows of one z line.  Within a group only the local row
// offsets k = 0..G-1 weight the densities in the field's precision (a0 = sum d,
// a1 = sum k d, a2 = sum k^2 d, and b0, b1 for the unit's last x); the base coordinates of
// the group (its first row Y_b, its line Z, the unit's first x X_0) multiply them in FP64:
//   sum Y d = Y_b a0 + s_y a1,  sum Y^2 d = Y_b^2 a0 + 2 Y_b s_y a1 + s_y^2 a2,
// so a rounding in a group is scaled by at most the group's extent.  The chain is taken as
// rows of R = 32 W sites (X = x_col + R row: the fold adds the row and column moments); its
// groups span G R sites, so in complex64 a0, a1, a2 are kept as FP32 pairs (two-sum, FMA
// product residual), exact to ~2^-48.
// One partial per block, folded in a fixed order: deterministic for a given geometry.
constexpr int kMom2 = 10;
constexpr int kMom2Group = 8;  // rows per group

struct Mom2Geo {
  int64_t units;    // units in all (ncoset * upc)
  int64_t upc;      // units per row of one coset
  int64_t rows;     // storage rows per coset (z, y), y fastest
  int64_t chunks;   // row chunks per unit
  int64_t rs;       // row stride (sites)
  int64_t cs;       // component stride (sites)
  int64_t coset;    // coset stride (sites)
  int64_t limit;    // sites per coset: an index r * rs + x at or past it is not a site (chain tail)
  int ny;           // rows per z line
  int sx, sy, sz;   // physical step per x, row and z line (sz = 0: no z axis)
  int bcc;          // physical coordinates offset by the coset index (2 m + c (1, 1, 1))
};

// Knuth's two-sum: s + e += p with the rounding error of s + p kept in e (FP32 pair sums).
__device__ __forceinline__ void ff_add(float& s, float& e, float p) {
  const float t = __fadd_rn(s, p);
  const float bb = __fsub_rn(t, s);
  e = __fadd_rn(e, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb)));
  s = t;
}
// s + e += k d, the product's rounding error from an FMA
__device__ __forceinline__ void ff_madd(float& s, float& e, float k, float d) {
  const float p = __fmul_rn(k, d);
  e = __fadd_rn(e, __fmaf_rn(k, d, -p));
  ff_add(s, e, p);
}

// S: spinor components; W: x per unit (2 only for complex64); FF: a0, a1, a2 as FP32 pairs
// (the chain in complex64, whose groups span G rows of R sites)
template <typename R, int S, int W, bool FF>
__global__ void __launch_bounds__(kObsThreads, 3) moments2_kernel(const typename Cplx<R>::T* __restrict__ psi,
                                                               Mom2Geo m, double* __restrict__ partials) {
  using C = typename Cplx<R>::T;
  using V = typename std::conditional<W == 2, float4, C>::type;
  constexpr int G = kMom2Group;
  constexpr int L = sizeof(V) == 16 ? 2 : 4;  // L S loads (128 B at S = 4) in flight per thread
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double acc[kMom2];
#pragma unroll
  for (int q = 0; q < kMom2; ++q) acc[q] = 0.0;
  if (t < m.units * m.chunks) {
    const int64_t j = t / m.units, u = t - j * m.units;
    const int c = u >= m.upc ? 1 : 0;
    const int64_t x = (u - c * m.upc) * W;
    const int off = m.bcc ? c : 0;
    // rows of this chunk; on the chain, rows past the last site of this unit hold nothing
    const int64_t rvalid = (m.limit - x + m.rs - 1) / m.rs;
    const int r0 = (int)(j * m.rows / m.chunks);
    int r1 = (int)((j + 1) * m.rows / m.chunks);
    if (r1 > rvalid) r1 = (int)rvalid;
    const C* col = psi + c * m.coset + x;
    const int64_t cs = m.cs / W, rs = m.rs;
    // per unit: N0 = sum d, N1 = sum d over the last x, SY = sum Y d, SY1 (last x), SYY,
    // SZ, SZ1 (last x), SZZ, SYZ
    double N0 = 0, N1 = 0, SY = 0, SY1 = 0, SYY = 0, SZ = 0, SZ1 = 0, SZZ = 0, SYZ = 0;
    const double sy = m.sy, sy2 = (double)m.sy * m.sy;
    int r = r0;
    int z = r0 / m.ny, y = r0 - z * m.ny;
    while (r < r1) {
      const int lend = r1 < r + (m.ny - y) ? r1 : r + (m.ny - y);  // end of this z line
      const double Zd = (double)(m.sz * z + off);
      for (; r < lend; r += G, y += G) {
        R a0 = 0, a1 = 0, a2 = 0, b0 = 0, b1 = 0;
        float e0 = 0.f, e1 = 0.f, e2 = 0.f;  // FF: the low parts of a0, a1, a2
#pragma unroll 1
        for (int k0 = 0; k0 < G; k0 += L) {  // not unrolled: L rows of loads in flight, not G
          V v[L][S];
#pragma unroll
          for (int l = 0; l < L; ++l) {
            const int rr = r + k0 + l;
            if (rr < lend) {
              const V* q = reinterpret_cast<const V*>(col + (int64_t)rr * rs);
#pragma unroll
              for (int s = 0; s < S; ++s) v[l][s] = q[s * cs];
            } else {
#pragma unroll
              for (int s = 0; s < S; ++s) v[l][s] = V{};
            }
          }
#pragma unroll
          for (int l = 0; l < L; ++l) {
            const R k = (R)(k0 + l);
            R d0 = 0, d1 = 0;
#pragma unroll
            for (int s = 0; s < S; ++s) {
              if constexpr (W == 2) {
                d0 = fmaf(v[l][s].x, v[l][s].x, fmaf(v[l][s].y, v[l][s].y, d0));
                d1 = fmaf(v[l][s].z, v[l][s].z, fmaf(v[l][s].w, v[l][s].w, d1));
              } else {
                d0 = fma(v[l][s].x, v[l][s].x, fma(v[l][s].y, v[l][s].y, d0));
              }
            }
            const R d = d0 + d1;
            if constexpr (FF) {
              ff_add(a0, e0, d);
              ff_madd(a1, e1, k, d);
              ff_madd(a2, e2, k * k, d);
            } else {
              a0 += d;
              a1 = fma(k, d, a1);
              a2 = fma(k * k, d, a2);
            }
            b0 += d1;
            b1 = fma(k, d1, b1);
          }
        }
        const double A0 = (double)a0 + e0, A1 = (double)a1 + e1, A2 = (double)a2 + e2, B0 = b0, B1 = b1;
        const double Yb = (double)(m.sy * y + off);
        const double ty = fma(sy, A1, Yb * A0);  // sum Y d over the group
        N0 += A0;
        N1 += B0;
        SY += ty;
        SY1 += fma(sy, B1, Yb * B0);
        SYY += fma(Yb, fma(2.0 * sy, A1, Yb * A0), sy2 * A2);
        SZ = fma(Zd, A0, SZ);
        SZ1 = fma(Zd, B0, SZ1);
        SZZ = fma(Zd * Zd, A0, SZZ);
        SYZ = fma(Zd, ty, SYZ);
      }
      r = lend;  // the next z line starts at y = 0
      y = 0;
      ++z;
    }
    // the unit's x are X0 and (W = 2) X0 + sx
    const double X0 = (double)(m.sx * x + off), sx = m.sx;
    acc[0] = N0;
    acc[1] = fma(X0, N0, sx * N1);
    acc[2] = SY;
    acc[3] = SZ;
    acc[4] = fma(X0 * X0, N0, (2.0 * X0 * sx + sx * sx) * N1);
    acc[5] = SYY;
    acc[6] = SZZ;
    acc[7] = fma(X0, SY, sx * SY1);
    acc[8] = fma(X0, SZ, sx * SZ1);
    acc[9] = SYZ;
  }
  block_sum<kMom2, kObsThreads>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < kMom2; ++q) partials[(int64_t)blockIdx.x * kMom2 + q] = acc[q];
  }
}

// merge_xy (the chain as rows of R sites): X = x_col + R row, so S_x = S_x' + S_y' and
// S_xx = S_x'x' + 2 S_x'y' + S_y'y', and the y moments are zero.
__global__ void __launch_bounds__(kObsThreads) fold_moments2_kernel(const double* __restrict__ partials, int nblk,
                                                                    int merge_xy, double* __restrict__ result) {
  double acc[kMom2];
#pragma unroll
  for (int j = 0; j < kMom2; ++j) acc[j] = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
#pragma unroll
    for (int j = 0; j < kMom2; ++j) acc[j] += partials[b * kMom2 + j];
  }
  block_sum<kMom2, kObsThreads>(acc);
  if (threadIdx.x == 0) {
    if (merge_xy) {
      acc[1] += acc[2];
      acc[4] += 2.0 * acc[7] + acc[5];
      acc[2] = acc[5] = acc[7] = 0.0;
    }
#pragma unroll
    for (int j = 0; j < kMom2; ++j) result[j] = acc[j];
  }
}

// Units x chunks threads, about one resident wave, at most kMom2MaxBlocks blocks (a unit is
// W x of a row; the chain's rows are R = 32 W sites).
template <typename R, int S, int W, bool FF = false>
static int launch_moments2_w(const Geometry& g, const void* psi, double* partials, cudaStream_t st) {
  using C = typename Cplx<R>::T;
  Mom2Geo m{};
  m.cs = g.vol;
  m.coset = (int64_t)g.s * g.vol;
  if (g.dim == 1) {
    m.rs = 32 * W;
    m.upc = 32;
    m.rows = (g.nx + m.rs - 1) / m.rs;
    m.ny = (int)m.rows;
    m.limit = g.nx;
    m.sx = 1;
    m.sy = (int)m.rs;
    m.sz = 0;
  } else {
    m.rs = g.nx;
    m.upc = g.nx / W;
    m.rows = g.nz * g.ny;
    m.ny = (int)g.ny;
    m.limit = m.rows * m.rs;
    m.sx = m.sy = g.dim == 3 ? 2 : 1;
    m.sz = g.dim == 3 ? 2 : 0;
  }
  m.bcc = g.dim == 3 ? 1 : 0;
  m.units = (int64_t)g.ncoset * m.upc;
  int64_t wave = (int64_t)resident_blocks(moments2_kernel<R, S, W, FF>, kObsThreads) * kObsThreads;
  if (wave <= 0) wave = (int64_t)kObsBlocks * kObsThreads;
  int64_t chunks = wave / m.units;
  const int64_t most = (m.rows + kMom2Group - 1) / kMom2Group;  // a chunk of G rows at least
  if (chunks > most) chunks = most;
  if (chunks > (int64_t)kMom2MaxBlocks * kObsThreads / m.units) chunks = (int64_t)kMom2MaxBlocks * kObsThreads / m.units;
  if (chunks < 1) chunks = 1;
  m.chunks = chunks;
  const int64_t blocks = (m.units * chunks + kObsThreads - 1) / kObsThreads;
  moments2_kernel<R, S, W, FF><<<(unsigned)blocks, kObsThreads, 0, st>>>(static_cast<const C*>(psi), m, partials);
  return (int)blocks;
}

template <typename R>
static int launch_moments2_t(const Geometry& g, const void* psi, double* partials, cudaStream_t st) {
  if constexpr (std::is_same<R, float>::value) {
    const bool pair = g.nx % 2 == 0 && aligned16(psi);
    if (g.dim == 1)  // s = 2
      return pair ? launch_moments2_w<R, 2, 2, true>(g, psi, partials, st)
                  : launch_moments2_w<R, 2, 1, true>(g, psi, partials, st);
    if (pair)
      return g.s == 2 ? launch_moments2_w<R, 2, 2>(g, psi, partials, st) : launch_moments2_w<R, 4, 2>(g, psi, partials, st);
  }
  return g.s == 2 ? launch_moments2_w<R, 2, 1>(g, psi, partials, st) : launch_moments2_w<R, 4, 1>(g, psi, partials, st);
}

qw_status launch_position_moments2(const Geometry& g, qw_dtype dt, const void* psi, double* partials,
                                   double* result, cudaStream_t st) {
  const int nblk = (dt == QW_C64) ? launch_moments2_t<float>(g, psi, partials, st)
                                  : launch_moments2_t<double>(g, psi, partials, st);
  QW_CHECK_LAUNCH("second moments launch");
  fold_moments2_kernel<<<1, kObsThreads, 0, st>>>(partials, nblk, g.dim == 1 ? 1 : 0, result);
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

// K sums over nblk partials [nblk][K], in a fixed order: CTA b of the grid folds the partials
// [b nblk / G, (b + 1) nblk / G) into out[b][K] (two chains per thread, then a block sum).
template <int K>
__global__ void __launch_bounds__(kObsThreads) fold_range_kernel(const double* __restrict__ partials, int64_t nblk,
                                                                 double* __restrict__ out) {
  const int64_t b0 = (int64_t)blockIdx.x * nblk / gridDim.x, b1 = ((int64_t)blockIdx.x + 1) * nblk / gridDim.x;
  double a0[K], a1[K];
#pragma unroll
  for (int q = 0; q < K; ++q) a0[q] = a1[q] = 0.0;
  int64_t b = b0 + threadIdx.x;
  for (; b + kObsThreads < b1; b += 2 * kObsThreads) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      a0[q] += partials[b * K + q];
      a1[q] += partials[(b + kObsThreads) * K + q];
    }
  }
  for (; b < b1; b += kObsThreads) {
#pragma unroll
    for (int q = 0; q < K; ++q) a0[q] += partials[b * K + q];
  }
  double acc[K];
#pragma unroll
  for (int q = 0; q < K; ++q) acc[q] = a0[q] + a1[q];
  block_sum<K, kObsThreads>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) out[(int64_t)blockIdx.x * K + q] = acc[q];
  }
}

qw_status launch_fold_partials(const double* partials, int64_t nblk, int K, double* stage, double* result,
                               cudaStream_t st) {
  if (K != 2 && K != 4) {
    set_error("fold of %d sums", K);
    return QW_EINVAL;
  }
  const bool two = nblk > 4 * kObsThreads;  // many partials: kFoldCtas CTAs first, then one
  const double* src = partials;
  int64_t n = nblk;
  if (two) {
    if (K == 2)
      fold_range_kernel<2><<<kFoldCtas, kObsThreads, 0, st>>>(partials, nblk, stage);
    else
      fold_range_kernel<4><<<kFoldCtas, kObsThreads, 0, st>>>(partials, nblk, stage);
    QW_CHECK_LAUNCH("fold launch");
    src = stage;
    n = kFoldCtas;
  }
  if (K == 2)
    fold_range_kernel<2><<<1, kObsThreads, 0, st>>>(src, n, result);
  else
    fold_range_kernel<4><<<1, kObsThreads, 0, st>>>(src, n, result);
  QW_CHECK_LAUNCH("fold launch");
  return QW_OK;
}

}  // namespace qw
