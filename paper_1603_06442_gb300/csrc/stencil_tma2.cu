// Two steps of the BCC update rule (Eq. upd-rule) per pass over HBM (complex64):
// temporal fusion of the TMA z-marching kernel.
//
// A CTA owns an x-y tile of 64 x TY2 cells of both cosets and walks a chunk of
// z-layers.  Per iteration i it holds in shared memory:
//   psi0 (input)  coset 0 and coset 1 at layers i, i+1 (plus layer i+2 in flight),
//                 each one TMA tensor copy of the box [x0-2, x0+66) x [y0-1, y0+TY2+1);
//   psi1 (after one step), computed here on the tile grown by the one-cell halo
//                 the second step needs:
//                   coset 1 at layer i   on x in [x0-1, x0+64), y in [y0-1, y0+TY2)
//                   coset 0 at layer i+1 on x in [x0, x0+65),   y in [y0, y0+TY2+1)
//                 (coset 1 at i-1 and coset 0 at i are kept from the previous iteration);
// and then writes psi2 = U psi1 at layer i of the tile to HBM.  The input box is the
// one the one-step kernel loads, so HBM sees one read and one write of the field per
// two steps; the cost is ~14% extra arithmetic on the halo ring.
// The kernel is bound by shared-memory bandwidth, so every thread computes two
// x-adjacent cells from three loaded columns and keeps, in registers, the
// components its next z-step reads again (pair_step), cutting shared-memory loads
// per cell by a third, and forms the neighbour sums in butterfly order (bcc_sums).
// Edge tiles get the periodic images of out-of-range cells as in the one-step kernel.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <vector>

#include "qw_internal.cuh"
#include "qw_tma.cuh"

namespace qw {
namespace zm2 {

using namespace zm;

constexpr int TY2 = 8, NT2 = 32 * TY2;      // tile rows, threads
constexpr int BY2 = TY2 + 2;                // box rows
constexpr int CS2 = BY2 * ROWF;             // floats per component
constexpr int BUF2_FLOATS = 4 * CS2;
constexpr int BUF2_BYTES = BUF2_FLOATS * 4;
constexpr int NS0 = 3;                      // psi0 ring per coset: layers i, i+1, i+2
constexpr int MAXF2 = 2;
constexpr int SMEM2_BYTES = (2 * NS0 + 4) * BUF2_BYTES + 2 * NS0 * 8 + 128;
static_assert(BUF2_BYTES % 128 == 0, "TMA destinations must stay 128-byte aligned");
static_assert(SMEM2_BYTES <= 227 * 1024, "shared memory budget");

// Three consecutive box cells [c0, c0 + 3) of one component row, c0 = 2 tx + OFF:
// an 8-byte and a 16-byte load (OFF odd) or a 16-byte and an 8-byte load (OFF even).
template <int OFF>
__device__ __forceinline__ Row3 srow_at(const float* row, int tx) {
  const float* p = row + 2 * (2 * tx + OFF);
  Row3 r;
  if constexpr (OFF % 2 == 1) {
    const float2 a = *reinterpret_cast<const float2*>(p);
    const float4 b = *reinterpret_cast<const float4*>(p + 2);
    r.lo = a;
    r.mid = make_float2(b.x, b.y);
    r.hi = make_float2(b.z, b.w);
  } else {
    const float4 a = *reinterpret_cast<const float4*>(p);
    const float2 b = *reinterpret_cast<const float2*>(p + 4);
    r.lo = make_float2(a.x, a.y);
    r.mid = make_float2(a.z, a.w);
    r.hi = b;
  }
  return r;
}

// psi1 rows are stored split by cell parity: the even cells (0, 2, ..., 66) of a row in
// floats [0, HALF), the odd cells in [HALF, 2 HALF).  A warp's three-cell windows of psi1
// then load as three 8-byte loads with consecutive addresses across the lanes (no bank
// conflicts), where the interleaved psi0 rows need an 8-byte load at a 16-byte lane stride.
constexpr int HALF = ROWF / 2;

// Cells [c0, c0 + 3) of one psi1 row, c0 = 2 tx + OFF (OFF = 1 or 2 in step 2).
template <int OFF>
__device__ __forceinline__ Row3 srow_eo(const float* row, int tx) {
  static_assert(OFF == 1 || OFF == 2, "psi1 windows start at an odd or even cell");
  const float2* ev = reinterpret_cast<const float2*>(row);
  const float2* od = reinterpret_cast<const float2*>(row + HALF);
  Row3 r;
  if constexpr (OFF == 2) {  // c0 = 2 (tx + 1)
    r.lo = ev[tx + 1];
    r.mid = od[tx + 1];
    r.hi = ev[tx + 2];
  } else {  // c0 = 2 tx + 1
    r.lo = od[tx];
    r.mid = ev[tx + 1];
    r.hi = od[tx + 1];
  }
  return r;
}

template <int OFF, bool EO>
__device__ __forceinline__ Row3 srow(const float* row, int tx) {
  if constexpr (EO)
    return srow_eo<OFF>(row, tx);
  else
    return srow_at<OFF>(row, tx);
}

// One step for the two cells of output coset C at box row R, box columns
// Q0 = 2 tx + QOFF and Q0 + 1 (QOFF even: 16-byte aligned).  Sources: the other
// coset at the h_z = +1 layer (la: components 0, 1, 3) and the h_z = -1 layer
// (lb: components 0, 1, 2), rows R - 1 + C (h_y = +1) and R + C (h_y = -1),
// columns Q0 - 1 + C .. Q0 + 1 + C; the mass term reads own (coset C).
//
// z-reuse: the h_z = -1 layer of this step is the h_z = +1 layer of the same
// thread's next step (one layer further in z), at the same rows and columns, and
// both read components 0 and 1 there.  carry keeps those two Row3 pairs in
// registers between the steps; with first = true they are loaded from la instead.
// EO: the sources are psi1 rows (parity-split layout) instead of psi0 rows.
template <int C, int QOFF, bool EO = false>
__device__ __forceinline__ void pair_step(Row3 (&carry)[2][2], bool first, const float* la, const float* lb,
                                          const float* own, int R, int tx, const Coef32& cf, float4 (&res)[4]) {
  constexpr int OFF = QOFF - 1 + C;
  Row3 d[2], a2[2], b2[2], c2[2];
#pragma unroll
  for (int iy = 0; iy < 2; ++iy) {
    const float* base = la + (R - 1 + C + iy) * ROWF;
    if (first) {
      carry[iy][0] = srow<OFF, EO>(base, tx);
      carry[iy][1] = srow<OFF, EO>(base + CS2, tx);
    }
    d[iy] = srow<OFF, EO>(base + 3 * CS2, tx);
    const float* bb = lb + (R - 1 + C + iy) * ROWF;
    a2[iy] = srow<OFF, EO>(bb, tx);
    b2[iy] = srow<OFF, EO>(bb + CS2, tx);
    c2[iy] = srow<OFF, EO>(bb + 2 * CS2, tx);
  }
  const Row3 a[2] = {carry[0][0], carry[1][0]}, b[2] = {carry[0][1], carry[1][1]};
  float2 S[2][4];
  bcc_sums<0>(S[0], a, b, d, a2, b2, c2);
  bcc_sums<1>(S[1], a, b, d, a2, b2, c2);
#pragma unroll
  for (int iy = 0; iy < 2; ++iy) {
    carry[iy][0] = a2[iy];
    carry[iy][1] = b2[iy];
  }
  float4 o[4];
  if constexpr (EO) {  // cells 2 tx + QOFF, + 1: even and odd halves of the row
    const float* ob = own + R * ROWF + 2 * (tx + QOFF / 2);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 e = *reinterpret_cast<const float2*>(ob + q * CS2);
      const float2 od = *reinterpret_cast<const float2*>(ob + q * CS2 + HALF);
      o[q] = make_float4(e.x, e.y, od.x, od.y);
    }
  } else {
    const float* ob = own + R * ROWF + 2 * (2 * tx + QOFF);
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = *reinterpret_cast<const float4*>(ob + q * CS2);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 w = o[q ^ 2];
    const float2 r0 = finish(cf, S[0][q], make_float2(w.x, w.y));
    const float2 r1 = finish(cf, S[1][q], make_float2(w.z, w.w));
    res[q] = make_float4(r0.x, r0.y, r1.x, r1.y);
  }
}

// psi1 cells 2 tx + QOFF (even) and 2 tx + QOFF + 1 (odd) of row R, parity-split layout.
template <int QOFF>
__device__ __forceinline__ void store_smem(float* dst, int R, int tx, const float4 (&res)[4]) {
  static_assert(QOFF % 2 == 0, "psi1 pairs start at an even cell");
  float* d = dst + R * ROWF + 2 * (tx + QOFF / 2);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    *reinterpret_cast<float2*>(d + q * CS2) = make_float2(res[q].x, res[q].y);
    *reinterpret_cast<float2*>(d + q * CS2 + HALF) = make_float2(res[q].z, res[q].w);
  }
}

// psi1 of both cosets on the region step 2 reads:
//   coset 1 at layer L1 on rows [0, TY2+1), columns [1, 66): pairs at Q0 = 2k, k < 33;
//   coset 0 at layer L1+1 on rows [1, TY2+2), columns [2, 67): pairs at Q0 = 2k + 2, k < 33.
// Thread (tx, ty) owns the pair k = tx of row ty (coset 1) and ty + 1 (coset 0),
// with z-reuse; the last row and the pair k = 32 of each coset (82 pairs) go to
// warps 0..3 without it, one kind per warp.
struct Step1Src {
  const float *c0a, *c0b, *c1a, *c1b;  // psi0 coset 0 / 1 at layers L1 (a) and L1 + 1 (b)
  float *p1c1, *p1c0;                  // psi1 destinations: coset 1 at L1, coset 0 at L1 + 1
};

// A thread's two psi1 pair results are written after both pair steps: the stores and the next
// pair's loads touch the same shared array, so the compiler keeps a store in order before them;
// with the stores last, both steps' loads can overlap (0.7% faster per launch at BCC N=512).
__device__ __forceinline__ void step1(const Step1Src& s, Row3 (&k1)[2][2], Row3 (&k0)[2][2], bool first,
                                      const Coef32& cf, int tx, int ty, int tid) {
  float4 res1[4], res0[4];
  // coset 1: la = coset 0 at L1 (h_z = +1), lb = coset 0 at L1 + 1, own coset 1 at L1
  pair_step<1, 0>(k1, first, s.c0a, s.c0b, s.c1a, ty, tx, cf, res1);
  // coset 0 at L1 + 1: la = coset 1 at L1, lb = coset 1 at L1 + 1, own coset 0 at L1 + 1
  pair_step<0, 2>(k0, first, s.c1a, s.c1b, s.c0b, ty + 1, tx, cf, res0);
  store_smem<0>(s.p1c1, ty, tx, res1);
  store_smem<2>(s.p1c0, ty + 1, tx, res0);
  // remainder, one warp per kind: warp 0 coset 1 row TY2, warp 1 coset 0 row TY2 + 1,
  // warp 2 coset 1 pair k = 32 of rows 0..TY2, warp 3 coset 0 pair k = 32 of rows 1..TY2+1
  const int w = tid >> 5;
  if (w < 2 || (w < 4 && tx <= TY2)) {
    Row3 tmp[2][2];
    const bool col = w >= 2;
    const int kk = col ? 32 : tx;
    if ((w & 1) == 0) {
      const int R = col ? tx : TY2;
      pair_step<1, 0>(tmp, true, s.c0a, s.c0b, s.c1a, R, kk, cf, res1);
      store_smem<0>(s.p1c1, R, kk, res1);
    } else {
      const int R = col ? tx + 1 : TY2 + 1;
      pair_step<0, 2>(tmp, true, s.c1a, s.c1b, s.c0b, R, kk, cf, res1);
      store_smem<2>(s.p1c0, R, kk, res1);
    }
  }
}

__global__ void __launch_bounds__(NT2, 1)
    step3d_c64_tma2_kernel(const __grid_constant__ CUtensorMap map, const float2* __restrict__ in,
                           float2* __restrict__ out, int M, const int4* __restrict__ items, int nitems, Coef32 cf,
                           int* err, int* next_item) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int s_item;
  unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  float* p0 = reinterpret_cast<float*>(smem);                // 2 * NS0 psi0 buffers: coset c, slot s -> c * NS0 + s
  float* p1 = p0 + 2 * NS0 * BUF2_FLOATS;                    // 4 psi1 buffers: coset c, slot s -> c * 2 + s
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (2 * NS0 + 4) * BUF2_BYTES);
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int64_t plane = (int64_t)M * M, vol = plane * M;
  const int tiles_x = M / TX;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(next_item, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= nitems) break;
    const int4 it = items[item];
    const int x0 = (it.x % tiles_x) * TX, y0 = (it.x / tiles_x) * TY2;
    const int zs = it.y, ze = it.z;

    FixT<MAXF2> fx;
    fix_setup<TY2, NT2, MAXF2>(fx, x0, y0, M, vol, tid, err);

    if (tid == 0) {
      for (int s = 0; s < 2 * NS0; ++s) mbar_init(&bars[s], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    auto wrapz = [&](int z) { return z < 0 ? z + M : (z >= M ? z - M : z); };
    auto slot0 = [&](int L) { return (L - (zs - 1)) % NS0; };
    auto par0 = [&](int L) { return (unsigned)(((L - (zs - 1)) / NS0) & 1); };
    auto buf0 = [&](int c, int L) { return p0 + (c * NS0 + slot0(L)) * BUF2_FLOATS; };
    auto bar0 = [&](int c, int L) { return &bars[c * NS0 + slot0(L)]; };
    auto buf1 = [&](int c, int L) {  // psi1 ring of two per coset
      const int s = (c == 1) ? ((L - (zs - 1)) & 1) : ((L - zs) & 1);
      return p1 + (c * 2 + s) * BUF2_FLOATS;
    };
    auto issue = [&](int c, int L) {
      uint64_t* b = bar0(c, L);
      mbar_expect_tx(b, BUF2_BYTES);
      tma_load_4d(buf0(c, L), &map, 2 * (x0 - 2), y0 - 1, wrapz(L), 4 * c, b);
    };
    auto fetch_fix = [&](int c, int L, float2 (&v)[MAXF2]) {
      const float2* base = in + (int64_t)c * 4 * vol + (int64_t)wrapz(L) * plane;
#pragma unroll
      for (int i = 0; i < MAXF2; ++i)
        if (i < fx.n) v[i] = __ldg(base + fx.goff[i]);
    };
    auto store_fix = [&](float* b, const float2 (&v)[MAXF2]) {
#pragma unroll
      for (int i = 0; i < MAXF2; ++i)
        if (i < fx.n) *reinterpret_cast<float2*>(b + fx.soff[i]) = v[i];
    };

    bool ok = true;
    float2 fA0[MAXF2], fA1[MAXF2], fB0[MAXF2], fB1[MAXF2], fC0[MAXF2], fC1[MAXF2];
    // prologue: psi0 layers zs-1, zs, zs+1 of both cosets; psi1 coset 1 at zs-1 and coset 0 at zs
    if (tid == 0) {
      fence_proxy_async();
      for (int L = zs - 1; L <= zs + 1; ++L) {
        issue(0, L);
        issue(1, L);
      }
    }
    fetch_fix(0, zs - 1, fB0);
    fetch_fix(1, zs - 1, fB1);
    fetch_fix(0, zs, fC0);
    fetch_fix(1, zs, fC1);
    fetch_fix(0, zs + 1, fA0);
    fetch_fix(1, zs + 1, fA1);
    ok &= mbar_wait(bar0(0, zs - 1), par0(zs - 1), err);
    ok &= mbar_wait(bar0(1, zs - 1), par0(zs - 1), err);
    ok &= mbar_wait(bar0(0, zs), par0(zs), err);
    ok &= mbar_wait(bar0(1, zs), par0(zs), err);
    store_fix(buf0(0, zs - 1), fB0);
    store_fix(buf0(1, zs - 1), fB1);
    store_fix(buf0(0, zs), fC0);
    store_fix(buf0(1, zs), fC1);
    ok = __syncthreads_and(ok);
    // z-reuse carries: step 1 (psi1 coset 1 / coset 0) and step 2 (output coset 0 / 1)
    Row3 k1[2][2], k0[2][2], q0[2][2], q1[2][2];
    if (ok) {
      const Step1Src s{buf0(0, zs - 1), buf0(0, zs), buf0(1, zs - 1), buf0(1, zs), buf1(1, zs - 1), buf1(0, zs)};
      step1(s, k1, k0, true, cf, tx, ty, tid);
    }
    __syncthreads();

    for (int i = zs; i < ze && ok; ++i) {
      const bool more = (i + 2 <= ze);
      if (more) {
        if (tid == 0) {
          fence_proxy_async();
          issue(0, i + 2);
          issue(1, i + 2);
        }
        fetch_fix(0, i + 2, fC0);
        fetch_fix(1, i + 2, fC1);
      }
      ok &= mbar_wait(bar0(0, i + 1), par0(i + 1), err);
      ok &= mbar_wait(bar0(1, i + 1), par0(i + 1), err);
      store_fix(buf0(0, i + 1), fA0);
      store_fix(buf0(1, i + 1), fA1);
      ok = __syncthreads_and(ok);
      if (!ok) break;
      // step 1: psi1 coset 1 at layer i, coset 0 at layer i+1
      {
        const Step1Src s{buf0(0, i), buf0(0, i + 1), buf0(1, i), buf0(1, i + 1), buf1(1, i), buf1(0, i + 1)};
        step1(s, k1, k0, false, cf, tx, ty, tid);
      }
      __syncthreads();
      // step 2: psi2 at layer i of the tile
      {
        const int64_t v4 = vol / 2;
        const int64_t orow = (int64_t)i * plane + (int64_t)(y0 + ty) * M + x0;
        float4* d0 = reinterpret_cast<float4*>(out + orow) + tx;
        float4* d1 = reinterpret_cast<float4*>(out + 4 * vol + orow) + tx;
        float4 res[4];
        pair_step<0, 2, true>(q0, i == zs, buf1(1, i - 1), buf1(1, i), buf1(0, i), ty + 1, tx, cf, res);
#pragma unroll
        for (int q = 0; q < 4; ++q) d0[q * v4] = res[q];
        pair_step<1, 2, true>(q1, i == zs, buf1(0, i), buf1(0, i + 1), buf1(1, i), ty + 1, tx, cf, res);
#pragma unroll
        for (int q = 0; q < 4; ++q) d1[q * v4] = res[q];
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < MAXF2; ++k) {
        fA0[k] = fC0[k];
        fA1[k] = fC1[k];
      }
    }
    if (!ok) {
      for (int k = 0; k < 1000; ++k) __nanosleep(1000);
      return;
    }
    __syncthreads();
  }
}

}  // namespace zm2

bool tma2_step_supported(const Geometry& g) {
  return g.dim == 3 && g.nx % zm::TX == 0 && g.nx % zm2::TY2 == 0 && g.nx >= zm::TX && g.nx <= 4096;
}

extern PFN_cuTensorMapEncodeTiled_v12000 tma_encoder();

qw_status launch_step_tma2(const Geometry& g, double n, double m, const void* in, void* out, const int4* items,
                           int nitems, int* err, int* next_item, cudaStream_t st) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tma_encoder();
  if (!enc) return QW_ECUDA;
  const int M = (int)g.nx;
  CUtensorMap map;
  cuuint64_t dims[4] = {(cuuint64_t)2 * M, (cuuint64_t)M, (cuuint64_t)M, 8};
  cuuint64_t strides[3] = {(cuuint64_t)2 * M * 4, (cuuint64_t)2 * M * M * 4, (cuuint64_t)2 * M * M * M * 4};
  cuuint32_t box[4] = {zm::ROWF, zm2::BY2, 1, 4};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(in), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return QW_ECUDA;
  }
  const qw_status sa = smem_attr(zm2::step3d_c64_tma2_kernel, zm2::SMEM2_BYTES);
  if (sa != QW_OK) return sa;
  int dev = 0, nsm = 0;
  QW_CHECK_CUDA(cudaGetDevice(&dev));
  QW_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int grid = nitems < nsm ? nitems : nsm;
  QW_CHECK_CUDA(cudaMemsetAsync(next_item, 0, sizeof(int), st));
  zm2::step3d_c64_tma2_kernel<<<grid, zm2::NT2, zm2::SMEM2_BYTES, st>>>(
      map, static_cast<const float2*>(in), static_cast<float2*>(out), M, items, nitems, make_coef32(3, n, m), err,
      next_item);
  QW_CHECK_LAUNCH("tma2 stencil launch");
  return QW_OK;
}

}  // namespace qw
