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

// One step for one cell of output coset C at box (row r, col q):
// la / lb = other coset at the h_z = +1 / -1 source layers, own = coset C at the output layer.
template <int HX, int HY, int HZ, int C>
__device__ __forceinline__ void cell_term(float2& S0, float2& S1, float2& S2, float2& S3, const float* lay, int r,
                                          int q) {
  constexpr int P = HX * HY * HZ;
  const int rr = (HY == 1) ? r - 1 + C : r + C;
  const int qq = (HX == 1) ? q - 1 + C : q + C;
  const float* base = lay + rr * ROWF + 2 * qq;
  if constexpr (HZ == 1) {
    const float2 a = *reinterpret_cast<const float2*>(base);
    const float2 b = *reinterpret_cast<const float2*>(base + CS2);
    const float2 d = *reinterpret_cast<const float2*>(base + 3 * CS2);
    cmac<1, -P>(S0, a);
    cmac<HX, -HY>(S0, b);
    cmac<-HX, HY>(S2, d);
    cmac<1, -P>(S3, d);
  } else {
    const float2 a = *reinterpret_cast<const float2*>(base);
    const float2 b = *reinterpret_cast<const float2*>(base + CS2);
    const float2 c = *reinterpret_cast<const float2*>(base + 2 * CS2);
    cmac<HX, HY>(S1, a);
    cmac<1, -P>(S1, b);
    cmac<1, -P>(S2, c);
    cmac<-HX, -HY>(S3, c);
  }
}

template <int C>
__device__ __forceinline__ void cell_step(const float* la, const float* lb, const float* own, float* dst, int r,
                                          int q, const Coef32& cf) {
  float2 S0 = make_float2(0.f, 0.f), S1 = S0, S2 = S0, S3 = S0;
  cell_term<+1, +1, +1, C>(S0, S1, S2, S3, la, r, q);
  cell_term<+1, -1, +1, C>(S0, S1, S2, S3, la, r, q);
  cell_term<-1, +1, +1, C>(S0, S1, S2, S3, la, r, q);
  cell_term<-1, -1, +1, C>(S0, S1, S2, S3, la, r, q);
  cell_term<+1, +1, -1, C>(S0, S1, S2, S3, lb, r, q);
  cell_term<+1, -1, -1, C>(S0, S1, S2, S3, lb, r, q);
  cell_term<-1, +1, -1, C>(S0, S1, S2, S3, lb, r, q);
  cell_term<-1, -1, -1, C>(S0, S1, S2, S3, lb, r, q);
  const int o = r * ROWF + 2 * q;
  const float2 o0 = *reinterpret_cast<const float2*>(own + o);
  const float2 o1 = *reinterpret_cast<const float2*>(own + o + CS2);
  const float2 o2 = *reinterpret_cast<const float2*>(own + o + 2 * CS2);
  const float2 o3 = *reinterpret_cast<const float2*>(own + o + 3 * CS2);
  *reinterpret_cast<float2*>(dst + o) = finish(cf, S0, o2);
  *reinterpret_cast<float2*>(dst + o + CS2) = finish(cf, S1, o3);
  *reinterpret_cast<float2*>(dst + o + 2 * CS2) = finish(cf, S2, o0);
  *reinterpret_cast<float2*>(dst + o + 3 * CS2) = finish(cf, S3, o1);
}

// psi1 of coset 1 on rows [0, TY2+1), cols [1, 66) and of coset 0 on rows [1, TY2+2), cols [2, 67).
__device__ __forceinline__ void step1(const float* c0a, const float* c0b, const float* c1a, const float* c1b,
                                      float* p1c1, float* p1c0, const Coef32& cf, int tid) {
  constexpr int W = TX + 1, CELLS = W * (TY2 + 1);
  // coset 1 at layer i: sources coset 0 at layers i (h_z = +1) and i+1, own coset 1 at i
  for (int k = tid; k < CELLS; k += NT2) {
    const int r = k / W, q = 1 + (k - (k / W) * W);
    cell_step<1>(c0a, c0b, c1a, p1c1, r, q, cf);
  }
  // coset 0 at layer i+1: sources coset 1 at layers i (h_z = +1) and i+1, own coset 0 at i+1
  for (int k = tid; k < CELLS; k += NT2) {
    const int r = 1 + k / W, q = 2 + (k - (k / W) * W);
    cell_step<0>(c1a, c1b, c0b, p1c0, r, q, cf);
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
    if (ok) {
      constexpr int W = TX + 1, CELLS = W * (TY2 + 1);
      for (int k = tid; k < CELLS; k += NT2) {
        const int r = k / W, q = 1 + (k - (k / W) * W);
        cell_step<1>(buf0(0, zs - 1), buf0(0, zs), buf0(1, zs - 1), buf1(1, zs - 1), r, q, cf);
      }
      for (int k = tid; k < CELLS; k += NT2) {
        const int r = 1 + k / W, q = 2 + (k - (k / W) * W);
        cell_step<0>(buf0(1, zs - 1), buf0(1, zs), buf0(0, zs), buf1(0, zs), r, q, cf);
      }
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
      step1(buf0(0, i), buf0(0, i + 1), buf0(1, i), buf0(1, i + 1), buf1(1, i), buf1(0, i + 1), cf, tid);
      __syncthreads();
      // step 2: psi2 at layer i of the tile
      {
        const int64_t v4 = vol / 2;
        const int64_t orow = (int64_t)i * plane + (int64_t)(y0 + ty) * M + x0;
        float4* d0 = reinterpret_cast<float4*>(out + orow) + tx;
        float4* d1 = reinterpret_cast<float4*>(out + 4 * vol + orow) + tx;
        compute<0, CS2>(buf1(1, i - 1), buf1(1, i), buf1(0, i), d0, v4, cf, tx, ty);
        compute<1, CS2>(buf1(0, i), buf1(0, i + 1), buf1(1, i), d1, v4, cf, tx, ty);
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
  static bool attr_done = false;
  if (!attr_done) {
    QW_CHECK_CUDA(cudaFuncSetAttribute(zm2::step3d_c64_tma2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       zm2::SMEM2_BYTES));
    attr_done = true;
  }
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
