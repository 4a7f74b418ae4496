// Probability projections (Sec. 5.2: the distribution of a localised state projected
// onto axes and planes): rho(x) = sum_s |psi_s(x)|^2 summed over the axes that are not
// kept, on the physical grid (lattice coordinates (a, b) in 2D, physical BCC
// coordinates 2 m + c (1, 1, 1) in 3D), in FP64.
//
// A storage row is the x line of one (coset, z, y).  An output row is a (coset, kept z,
// kept y); its reduced rows are the (z, y) that match it.  Two kernels:
//   x kept    a thread owns one x of an output row and a chunk of its reduced rows
//             (the threads of a warp read consecutive x);
//   x summed  a warp owns an output row and a chunk of its reduced rows, lanes striding
//             along x, then a warp sum.
// With one chunk a kernel writes the physical output directly; otherwise it writes
// partials [chunk][output] and a fold adds the chunks in a fixed order (a thread per output,
// or with 64 chunks or more a warp per output).  Site densities
// are taken in the field's precision and summed in FP64 in a fixed order: deterministic.
#include <cuda_runtime.h>

#include "qw_internal.cuh"

namespace qw {
namespace {

struct ProjGeo {
  int dim, s, ncos, N;
  int nx, ny, nz;
  int kx, ky, kz;        // kept axes
  int oy, oz;            // output-row extents: ny or 1, nz or 1
  int ry;                // reduced-row extent along y: 1 (kept) or ny
  int chunks;
  int pair;              // x kept, complex64, nx even: a thread owns two adjacent x (16-byte loads)
  int64_t vol;
  int64_t n_orows;       // ncos * oz * oy
  int64_t rrows;         // reduced rows per output row
  int64_t nout;          // storage outputs: n_orows * (kx ? nx : 1)
};

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

__device__ __forceinline__ void decode_orow(const ProjGeo& p, int64_t orow, int& c, int& zk, int& yk) {
  yk = (int)(orow % p.oy);
  const int64_t t = orow / p.oy;
  zk = (int)(t % p.oz);
  c = (int)(t / p.oz);
}

// Physical output index of storage output (c, zk, yk, xk): x fastest, then y, then z
// among the kept axes.
__device__ __forceinline__ int64_t phys_index(const ProjGeo& p, int c, int zk, int yk, int xk) {
  const int sc = p.dim == 3 ? 2 : 1, off = p.dim == 3 ? c : 0;
  int64_t idx = 0, mul = 1;
  if (p.kx) {
    idx += (int64_t)(sc * xk + off);
    mul = p.N;
  }
  if (p.ky) {
    idx += (int64_t)(sc * yk + off) * mul;
    mul *= p.N;
  }
  if (p.kz) idx += (int64_t)(sc * zk + off) * mul;
  return idx;
}

template <typename R>
__device__ __forceinline__ R density(const typename Cx<R>::T* __restrict__ q, int s, int64_t vol) {
  R d = 0;
  for (int j = 0; j < s; ++j) {
    const typename Cx<R>::T v = q[(int64_t)j * vol];
    d = fma(v.x, v.x, d);
    d = fma(v.y, v.y, d);
  }
  return d;
}

// Walks the storage rows (c, z, y) of reduced rows r0, r0 + 1, ... of output row
// (c, zk, yk) without a division per row.
struct RowWalk {
  int z, y;
  __device__ RowWalk(const ProjGeo& p, int zk, int yk, int64_t r0) {
    z = p.kz ? zk : (int)(r0 / p.ry);
    y = p.ky ? yk : (int)(r0 % p.ry);
  }
  __device__ __forceinline__ int64_t offset(const ProjGeo& p, int c) const {
    return (int64_t)c * p.s * p.vol + ((int64_t)z * p.ny + y) * p.nx;
  }
  __device__ __forceinline__ void next(const ProjGeo& p) {
    if (!p.ky && ++y < p.ny) return;
    y = p.ky ? y : 0;
    ++z;  // z is not kept here: a kept z has one reduced row per y
  }
};

// S: spinor components, G: rows per group (4, or 1 when a chunk has fewer than four rows),
// compile time: a group's loads (G rows, every component) are all issued before its sums.
template <typename R, int S, int G>
__global__ void __launch_bounds__(256) proj_x_kernel(const typename Cx<R>::T* __restrict__ psi, ProjGeo p,
                                                     double* __restrict__ out, double* __restrict__ partials) {
  using C = typename Cx<R>::T;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= p.nout) return;
  const int x = (int)(gid % p.nx);
  const int64_t orow = gid / p.nx;
  int c, zk, yk;
  decode_orow(p, orow, c, zk, yk);
  const int j = blockIdx.y;
  const int64_t r0 = j * p.rrows / p.chunks, r1 = (j + 1) * p.rrows / p.chunks;
  double acc = 0.0;
  RowWalk w(p, zk, yk, r0);
  // groups of G rows summed in the field's precision, then in FP64
  for (int64_t r = r0; r < r1; r += G) {
    C v[G][S];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      if (r + u < r1) {
        const C* q = psi + w.offset(p, c) + x;
#pragma unroll
        for (int k = 0; k < S; ++k) v[u][k] = q[(int64_t)k * p.vol];
        w.next(p);
      } else {
#pragma unroll
        for (int k = 0; k < S; ++k) v[u][k] = C{0, 0};
      }
    }
    R g = 0;
#pragma unroll
    for (int u = 0; u < G; ++u)
#pragma unroll
      for (int k = 0; k < S; ++k) g = fma(v[u][k].x, v[u][k].x, fma(v[u][k].y, v[u][k].y, g));
    acc += (double)g;
  }
  if (p.chunks == 1)
    out[phys_index(p, c, zk, yk, x)] = acc;
  else
    partials[(int64_t)j * p.nout + gid] = acc;
}

// proj_x_kernel for complex64 with two adjacent x per thread (x even): one 16-byte load per
// component and row instead of two 8-byte ones.
template <int S, int G>
__global__ void __launch_bounds__(256) proj_x2_kernel(const float2* __restrict__ psi, ProjGeo p,
                                                      double* __restrict__ out, double* __restrict__ partials) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= p.nout / 2) return;
  const int64_t o = 2 * gid;
  const int x = (int)(o % p.nx);
  const int64_t orow = o / p.nx;
  int c, zk, yk;
  decode_orow(p, orow, c, zk, yk);
  const int j = blockIdx.y;
  const int64_t r0 = j * p.rrows / p.chunks, r1 = (j + 1) * p.rrows / p.chunks;
  double a0 = 0.0, a1 = 0.0;
  RowWalk w(p, zk, yk, r0);
  for (int64_t r = r0; r < r1; r += G) {
    float4 v[G][S];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      if (r + u < r1) {
        const float2* q = psi + w.offset(p, c) + x;
#pragma unroll
        for (int k = 0; k < S; ++k) v[u][k] = *reinterpret_cast<const float4*>(q + (int64_t)k * p.vol);
        w.next(p);
      } else {
#pragma unroll
        for (int k = 0; k < S; ++k) v[u][k] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    float g0 = 0.f, g1 = 0.f;
#pragma unroll
    for (int u = 0; u < G; ++u)
#pragma unroll
      for (int k = 0; k < S; ++k) {
        g0 = fmaf(v[u][k].x, v[u][k].x, fmaf(v[u][k].y, v[u][k].y, g0));
        g1 = fmaf(v[u][k].z, v[u][k].z, fmaf(v[u][k].w, v[u][k].w, g1));
      }
    a0 += (double)g0;
    a1 += (double)g1;
  }
  if (p.chunks == 1) {
    out[phys_index(p, c, zk, yk, x)] = a0;
    out[phys_index(p, c, zk, yk, x + 1)] = a1;
  } else {
    partials[(int64_t)j * p.nout + o] = a0;
    partials[(int64_t)j * p.nout + o + 1] = a1;
  }
}

// BCC, every axis kept (the site density on the physical N^3 grid): a thread owns W cells
// of one storage x line and the 2 W physical points (2 x, 2 x + 1, ...) of one physical row
// (Z, Y), which it writes whole: the density at the even points of a row with Z and Y even
// (coset 0), at the odd points of a row with Z and Y odd (coset 1), zero elsewhere (rows of
// mixed parity are written without a read).  V2: out is 16-byte aligned.
template <typename R, int W, bool V2>
__global__ void __launch_bounds__(256) density_bcc_kernel(const typename Cx<R>::T* __restrict__ psi, ProjGeo p,
                                                          double* __restrict__ out) {
  using C = typename Cx<R>::T;
  const int64_t per_row = p.nx / W;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)p.N * p.N * per_row) return;
  const int64_t prow = gid / per_row;  // Z * N + Y
  const int xi = (int)(gid - prow * per_row) * W;
  const int Z = (int)(prow / p.N), Y = (int)(prow - (int64_t)Z * p.N);
  double d[W];
#pragma unroll
  for (int w = 0; w < W; ++w) d[w] = 0.0;
  const int c = Z & 1;
  const bool site = (Z & 1) == (Y & 1);
  if (site) {
    const C* q = psi + (int64_t)c * p.s * p.vol + ((int64_t)(Z >> 1) * p.ny + (Y >> 1)) * p.nx + xi;
    if constexpr (W == 2) {
      float4 v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = *reinterpret_cast<const float4*>(q + (int64_t)k * p.vol);
      float g0 = 0.f, g1 = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        g0 = fmaf(v[k].x, v[k].x, fmaf(v[k].y, v[k].y, g0));
        g1 = fmaf(v[k].z, v[k].z, fmaf(v[k].w, v[k].w, g1));
      }
      d[0] = g0;
      d[W - 1] = g1;
    } else {
      C v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = q[(int64_t)k * p.vol];
      R g = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) g = fma(v[k].x, v[k].x, fma(v[k].y, v[k].y, g));
      d[0] = (double)g;
    }
  }
  double* o = out + prow * p.N + 2 * xi;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const double e = c ? 0.0 : d[w], f = c ? d[w] : 0.0;  // points 2 (xi + w) and 2 (xi + w) + 1
    if constexpr (V2) {
      *reinterpret_cast<double2*>(o + 2 * w) = make_double2(e, f);
    } else {
      o[2 * w] = e;
      o[2 * w + 1] = f;
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(256) proj_w_kernel(const typename Cx<R>::T* __restrict__ psi, ProjGeo p,
                                                     double* __restrict__ out, double* __restrict__ partials) {
  const int64_t orow = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (orow >= p.n_orows) return;  // whole warps leave together
  int c, zk, yk;
  decode_orow(p, orow, c, zk, yk);
  const int j = blockIdx.y;
  const int64_t r0 = j * p.rrows / p.chunks, r1 = (j + 1) * p.rrows / p.chunks;
  double acc = 0.0;
  RowWalk w(p, zk, yk, r0);
  for (int64_t r = r0; r < r1; ++r) {
    const typename Cx<R>::T* row = psi + w.offset(p, c);
    R g = 0;
    for (int x = lane; x < p.nx; x += 32) g += density<R>(row + x, p.s, p.vol);
    acc += (double)g;
    w.next(p);
  }
  acc = warp_sum_d(acc);
  if (lane == 0) {
    if (p.chunks == 1)
      out[phys_index(p, c, zk, yk, 0)] = acc;
    else
      partials[(int64_t)j * p.n_orows + orow] = acc;
  }
}

__global__ void __launch_bounds__(256) proj_fold_kernel(const double* __restrict__ partials, ProjGeo p,
                                                        double* __restrict__ out) {
  const int64_t nout = p.kx ? p.nout : p.n_orows;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nout) return;
  double acc = 0.0;
  for (int j = 0; j < p.chunks; ++j) acc += partials[(int64_t)j * nout + gid];
  const int xk = p.kx ? (int)(gid % p.nx) : 0;
  const int64_t orow = p.kx ? gid / p.nx : gid;
  int c, zk, yk;
  decode_orow(p, orow, c, zk, yk);
  out[phys_index(p, c, zk, yk, xk)] = acc;
}

// proj_fold_kernel for many chunks (few outputs, each with a long column of partials): a warp
// per output, lane l adding the chunks l, l + 32, ..., then a warp sum (a fixed order).
__global__ void __launch_bounds__(256) proj_fold_warp_kernel(const double* __restrict__ partials, ProjGeo p,
                                                             double* __restrict__ out) {
  const int64_t nout = p.kx ? p.nout : p.n_orows;
  const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gid >= nout) return;  // whole warps leave together
  double acc = 0.0;
  for (int j = lane; j < p.chunks; j += 32) acc += partials[(int64_t)j * nout + gid];
  acc = warp_sum_d(acc);
  if (lane == 0) {
    const int xk = p.kx ? (int)(gid % p.nx) : 0;
    const int64_t orow = p.kx ? gid / p.nx : gid;
    int c, zk, yk;
    decode_orow(p, orow, c, zk, yk);
    out[phys_index(p, c, zk, yk, xk)] = acc;
  }
}

// Threads (x kept) and warps (x summed) a launch aims for: ~1700 threads per SM.
constexpr int64_t kProjThreads = int64_t(1) << 18;
constexpr int64_t kProjWarps = kProjThreads / 32;

// al16: the field is 16-byte aligned (complex64 pairs of x are loaded as one vector).  The
// partial count with al16 = true bounds the one without (pairs halve the work units).
ProjGeo make_proj(const Geometry& g, int keep, qw_dtype dt, bool al16 = true) {
  ProjGeo p{};
  p.dim = g.dim;
  p.s = g.s;
  p.ncos = g.ncoset;
  p.N = (int)g.N;
  p.nx = (int)g.nx;
  p.ny = (int)g.ny;
  p.nz = (int)g.nz;
  p.kx = keep & 1;
  p.ky = (keep >> 1) & 1;
  p.kz = (keep >> 2) & 1;
  p.oy = p.ky ? p.ny : 1;
  p.oz = p.kz ? p.nz : 1;
  p.ry = p.ky ? 1 : p.ny;
  p.vol = g.vol;
  p.n_orows = (int64_t)p.ncos * p.oz * p.oy;
  p.rrows = (int64_t)(p.kz ? 1 : p.nz) * p.ry;
  p.nout = p.n_orows * (p.kx ? p.nx : 1);
  p.pair = (p.kx && dt == QW_C64 && p.nx % 2 == 0 && al16) ? 1 : 0;
  const int64_t units = p.kx ? (p.pair ? p.nout / 2 : p.nout) : p.n_orows;
  const int64_t want = p.kx ? kProjThreads : kProjWarps;
  int64_t k = (want + units - 1) / units;
  if (k > p.rrows) k = p.rrows;
  if (k > 65535) k = 65535;
  p.chunks = (int)(k < 1 ? 1 : k);
  return p;
}

}  // namespace

int64_t projection_partials(const Geometry& g, int keep, qw_dtype dt) {
  const ProjGeo p = make_proj(g, keep, dt);
  return p.chunks == 1 ? 0 : (int64_t)p.chunks * (p.kx ? p.nout : p.n_orows);
}

int64_t projection_outputs(const Geometry& g, int keep) {
  int64_t n = 1;
  for (int a = 0; a < 3; ++a)
    if ((keep >> a) & 1) n *= g.N;
  return n;
}

qw_status launch_projection(const Geometry& g, qw_dtype dt, const void* psi, int keep, double* out,
                            double* partials, cudaStream_t st) {
  const ProjGeo p = make_proj(g, keep, dt, aligned16(psi));
  const int kept = p.kx + p.ky + p.kz;
  if (g.dim == 3 && kept == 3) {  // every point of the output written once, zeros included
    const int w = p.pair ? 2 : 1;
    const int64_t threads = (int64_t)p.N * p.N * (p.nx / w);
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    const bool v2 = aligned16(out);
    if (dt == QW_C64 && p.pair)
      v2 ? density_bcc_kernel<float, 2, true><<<blocks, 256, 0, st>>>(static_cast<const float2*>(psi), p, out)
         : density_bcc_kernel<float, 2, false><<<blocks, 256, 0, st>>>(static_cast<const float2*>(psi), p, out);
    else if (dt == QW_C64)
      v2 ? density_bcc_kernel<float, 1, true><<<blocks, 256, 0, st>>>(static_cast<const float2*>(psi), p, out)
         : density_bcc_kernel<float, 1, false><<<blocks, 256, 0, st>>>(static_cast<const float2*>(psi), p, out);
    else
      v2 ? density_bcc_kernel<double, 1, true><<<blocks, 256, 0, st>>>(static_cast<const double2*>(psi), p, out)
         : density_bcc_kernel<double, 1, false><<<blocks, 256, 0, st>>>(static_cast<const double2*>(psi), p, out);
    QW_CHECK_LAUNCH("density launch");
    return QW_OK;
  }
  // BCC: physical points of mixed coordinate parity are not sites (two or more kept axes)
  if (g.dim == 3 && kept >= 2)
    QW_CHECK_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * projection_outputs(g, keep), st));
  const int64_t threads = p.kx ? (p.pair ? p.nout / 2 : p.nout) : p.n_orows * 32;
  const dim3 grid((unsigned)((threads + 255) / 256), (unsigned)p.chunks);
  const bool few = p.rrows < 4 * (int64_t)p.chunks;  // chunks of fewer than four rows: one row per group
  if (p.pair) {
    const float2* q = static_cast<const float2*>(psi);
    if (g.s == 2)
      few ? proj_x2_kernel<2, 1><<<grid, 256, 0, st>>>(q, p, out, partials)
          : proj_x2_kernel<2, 4><<<grid, 256, 0, st>>>(q, p, out, partials);
    else
      few ? proj_x2_kernel<4, 1><<<grid, 256, 0, st>>>(q, p, out, partials)
          : proj_x2_kernel<4, 4><<<grid, 256, 0, st>>>(q, p, out, partials);
  } else if (p.kx && dt == QW_C64) {
    const float2* q = static_cast<const float2*>(psi);
    if (g.s == 2)
      few ? proj_x_kernel<float, 2, 1><<<grid, 256, 0, st>>>(q, p, out, partials)
          : proj_x_kernel<float, 2, 4><<<grid, 256, 0, st>>>(q, p, out, partials);
    else
      few ? proj_x_kernel<float, 4, 1><<<grid, 256, 0, st>>>(q, p, out, partials)
          : proj_x_kernel<float, 4, 4><<<grid, 256, 0, st>>>(q, p, out, partials);
  } else if (p.kx) {
    const double2* q = static_cast<const double2*>(psi);
    if (g.s == 2)
      few ? proj_x_kernel<double, 2, 1><<<grid, 256, 0, st>>>(q, p, out, partials)
          : proj_x_kernel<double, 2, 4><<<grid, 256, 0, st>>>(q, p, out, partials);
    else
      few ? proj_x_kernel<double, 4, 1><<<grid, 256, 0, st>>>(q, p, out, partials)
          : proj_x_kernel<double, 4, 4><<<grid, 256, 0, st>>>(q, p, out, partials);
  } else {
    if (dt == QW_C64)
      proj_w_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float2*>(psi), p, out, partials);
    else
      proj_w_kernel<double><<<grid, 256, 0, st>>>(static_cast<const double2*>(psi), p, out, partials);
  }
  QW_CHECK_LAUNCH("projection launch");
  if (p.chunks > 1) {
    const int64_t n = p.kx ? p.nout : p.n_orows;
    if (p.chunks >= 64)
      proj_fold_warp_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(partials, p, out);
    else
      proj_fold_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(partials, p, out);
    QW_CHECK_LAUNCH("projection fold launch");
  }
  return QW_OK;
}

}  // namespace qw
