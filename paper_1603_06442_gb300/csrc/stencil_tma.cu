// BCC stencil step (Eq. upd-rule) for complex64, z-marching with TMA-staged tiles.
//
// Same arithmetic as the vectorised kernel of stencil.cu (transition matrices
// derived there); only the data movement differs.  A CTA owns an x-y tile of
// TX x TY cells of both cosets and walks a chunk of z-layers:
//   output coset 0 at layer z reads coset 1 at layers z-1 (h_z = +1) and z,
//   output coset 1 at layer z reads coset 0 at layers z (h_z = +1) and z+1,
// so each coset-layer is brought into shared memory once by one TMA tensor copy
// (all four components, box [x0-2, x0+TX+2) x [y0-1, y0+TY+1)) and used by two
// consecutive iterations.  The copies of the next two layer pairs are in flight
// while the current one is computed (mbarrier completion, bounded waits).
// Cells outside [0, M) of an edge tile are zero-filled by the TMA unit and then
// overwritten with their periodic images (loaded one iteration ahead).
// Algorithmic traffic: one read and one write of the field per step; halo rows
// and columns are re-read by the neighbouring tile, normally from L2.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <vector>

#include "qw_internal.cuh"
#include "qw_tma.cuh"

namespace qw {
namespace zm {

constexpr int TY = 4, NT = 128;           // tile rows, threads: 32 x 4
constexpr int BY = TY + 2;                // box rows: [y0 - 1, y0 + TY + 1)
constexpr int CSTR = BY * ROWF;           // floats per component
constexpr int BUF_FLOATS = 4 * CSTR;
constexpr int BUF_BYTES = BUF_FLOATS * 4;
constexpr int NSLOT = 4;                  // ring depth per coset: two layer pairs in flight
constexpr int MAX_FIX = 3;                // periodic-image cells per thread per buffer
constexpr int SMEM_BYTES = 2 * NSLOT * BUF_BYTES + 2 * NSLOT * 8 + 128;  // + alignment slack

static_assert(BUF_BYTES % 128 == 0, "TMA destinations must stay 128-byte aligned");
static_assert(ROWF <= 256 && BY <= 256, "TMA box extents");

__global__ void __launch_bounds__(NT, 2)
    step3d_c64_tma_kernel(const __grid_constant__ CUtensorMap map, const float2* __restrict__ in,
                          float2* __restrict__ out, int M, const int4* __restrict__ items, int nitems, Coef32 cf,
                          int* err, int* next_item) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int s_item;
  // TMA destinations must be 128-byte aligned: align the dynamic block by hand
  unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  float* buf = reinterpret_cast<float*>(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * NSLOT * BUF_BYTES);
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int64_t plane = (int64_t)M * M, vol = plane * M;
  const int tiles_x = M / TX;

  for (;;) {
    // dynamic schedule over a guided item table (long z-chunks first, short
    // ones last): few pipeline restarts and a short tail
    if (tid == 0) s_item = atomicAdd(next_item, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= nitems) break;
    const int4 it = items[item];
    const int tile = it.x;
    const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
    const int zs = it.y, ze = it.z;

    FixT<MAX_FIX> fx;
    fix_setup<TY, NT, MAX_FIX>(fx, x0, y0, M, vol, tid, err);

    if (tid == 0) {
      for (int s = 0; s < 2 * NSLOT; ++s) mbar_init(&bars[s], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // ring slots: coset c, layer L -> slot index into bars/buf
    auto slot1 = [&](int L) { return NSLOT + ((L - (zs - 1)) % NSLOT); };      // coset 1, L >= zs - 1
    auto slot0 = [&](int L) { return (L - zs) % NSLOT; };                    // coset 0, L >= zs
    auto par1 = [&](int L) { return (unsigned)(((L - (zs - 1)) / NSLOT) & 1); };
    auto par0 = [&](int L) { return (unsigned)(((L - zs) / NSLOT) & 1); };
    auto wrapz = [&](int z) { return z < 0 ? z + M : (z >= M ? z - M : z); };
    auto issue = [&](int slot, int coset, int L) {
      uint64_t* b = &bars[slot];
      mbar_expect_tx(b, BUF_BYTES);
      tma_load_4d(buf + slot * BUF_FLOATS, &map, 2 * (x0 - 2), y0 - 1, wrapz(L), 4 * coset, b);
    };
    auto fetch_fix = [&](int coset, int L, float2 (&v)[MAX_FIX]) {
      const float2* base = in + (int64_t)coset * 4 * vol + (int64_t)wrapz(L) * plane;
#pragma unroll
      for (int i = 0; i < MAX_FIX; ++i)
        if (i < fx.n) v[i] = __ldg(base + fx.goff[i]);
    };
    auto store_fix = [&](int slot, const float2 (&v)[MAX_FIX]) {
      float* b = buf + slot * BUF_FLOATS;
#pragma unroll
      for (int i = 0; i < MAX_FIX; ++i)
        if (i < fx.n) *reinterpret_cast<float2*>(b + fx.soff[i]) = v[i];
    };

    // fix-up registers: A = pair waited on this iteration, B = next, C = fetched now
    float2 f1a[MAX_FIX], f0a[MAX_FIX], f1b[MAX_FIX], f0b[MAX_FIX], f1c[MAX_FIX], f0c[MAX_FIX];
    bool ok = true;
    // prologue: coset 1 layers zs-1 .. zs+1, coset 0 layers zs .. zs+2
    const bool two = (zs + 1 < ze);
    if (tid == 0) {
      fence_proxy_async();
      issue(slot1(zs - 1), 1, zs - 1);
      issue(slot0(zs), 0, zs);
      issue(slot1(zs), 1, zs);
      issue(slot0(zs + 1), 0, zs + 1);
      if (two) {
        issue(slot1(zs + 1), 1, zs + 1);
        issue(slot0(zs + 2), 0, zs + 2);
      }
    }
    fetch_fix(1, zs - 1, f1c);
    fetch_fix(0, zs, f0c);
    fetch_fix(1, zs, f1a);
    fetch_fix(0, zs + 1, f0a);
    if (two) {
      fetch_fix(1, zs + 1, f1b);
      fetch_fix(0, zs + 2, f0b);
    }
    ok &= mbar_wait(&bars[slot1(zs - 1)], par1(zs - 1), err);
    ok &= mbar_wait(&bars[slot0(zs)], par0(zs), err);
    store_fix(slot1(zs - 1), f1c);
    store_fix(slot0(zs), f0c);
    ok = __syncthreads_and(ok);

    for (int z = zs; z < ze && ok; ++z) {
      // prefetch two layer pairs ahead: coset 1 layer z+2, coset 0 layer z+3
      const bool more = (z + 2 < ze);
      if (more) {
        if (tid == 0) {
          fence_proxy_async();
          issue(slot1(z + 2), 1, z + 2);
          issue(slot0(z + 3), 0, z + 3);
        }
        fetch_fix(1, z + 2, f1c);
        fetch_fix(0, z + 3, f0c);
      }
      ok &= mbar_wait(&bars[slot1(z)], par1(z), err);
      ok &= mbar_wait(&bars[slot0(z + 1)], par0(z + 1), err);
      store_fix(slot1(z), f1a);
      store_fix(slot0(z + 1), f0a);
      ok = __syncthreads_and(ok);
      if (ok) {
        const int64_t v4 = vol / 2;
        const int64_t orow = (int64_t)z * plane + (int64_t)(y0 + ty) * M + x0;
        float4* d0 = reinterpret_cast<float4*>(out + orow) + tx;
        float4* d1 = reinterpret_cast<float4*>(out + 4 * vol + orow) + tx;
        const float* c1m = buf + slot1(z - 1) * BUF_FLOATS;
        const float* c1z = buf + slot1(z) * BUF_FLOATS;
        const float* c0z = buf + slot0(z) * BUF_FLOATS;
        const float* c0p = buf + slot0(z + 1) * BUF_FLOATS;
        compute<0, CSTR>(c1m, c1z, c0z, d0, v4, cf, tx, ty);
        compute<1, CSTR>(c0z, c0p, c1z, d1, v4, cf, tx, ty);
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < MAX_FIX; ++i) {
        f1a[i] = f1b[i];
        f0a[i] = f0b[i];
        f1b[i] = f1c[i];
        f0b[i] = f0c[i];
      }
    }
    if (!ok) {
      // a copy never landed: give the ones still in flight a bounded time
      // (about a millisecond) to finish before the CTA leaves
      for (int i = 0; i < 1000; ++i) __nanosleep(1000);
      return;
    }
    __syncthreads();
  }
}

}  // namespace zm

// The driver's tensor-map encoder, looked up once (thread-safe static initialisation).
static PFN_cuTensorMapEncodeTiled_v12000 lookup_encoder() {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return nullptr;
  return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
}

PFN_cuTensorMapEncodeTiled_v12000 tma_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 enc = lookup_encoder();
  if (!enc) set_error("cuTensorMapEncodeTiled unavailable");
  return enc;
}

bool tma_step_supported(const Geometry& g) {
  return g.dim == 3 && g.nx % zm::TX == 0 && g.nx >= zm::TX && g.nx <= 4096;
}

std::vector<int4> tma_item_table(const Geometry& g, int resident, int ty) {
  // Every tile's z-range is cut the same way: chunks of 64 layers while more
  // than a quarter of the box remains, then halving down to 8.  Items are
  // ordered chunk by chunk over all tiles, so the short chunks come last (the
  // tail of the dynamic schedule) and running CTAs work on neighbouring tiles
  // at similar depths (shared halo rows stay in L2).
  const int M = (int)g.nx;
  const int ntiles = (M / zm::TX) * (M / ty);
  std::vector<int> cuts;  // chunk boundaries
  int z = 0;
  while (z < M) {
    const int rem = M - z;
    int c = 64;
    while (c > 8 && (c > rem || (int64_t)ntiles * rem < (int64_t)resident * c)) c /= 2;
    if (c > rem) c = rem;
    cuts.push_back(z);
    z += c;
  }
  cuts.push_back(M);
  std::vector<int4> items;
  for (size_t k = 0; k + 1 < cuts.size(); ++k)
    for (int t = 0; t < ntiles; ++t) items.push_back(make_int4(t, cuts[k], cuts[k + 1], 0));
  return items;
}

qw_status launch_step_tma(const Geometry& g, double n, double m, const void* in, void* out, const int4* items,
                          int nitems, int* err, int* next_item, cudaStream_t st) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tma_encoder();
  if (!enc) return QW_ECUDA;
  qw_status s;
  const int M = (int)g.nx;
  CUtensorMap map;
  cuuint64_t dims[4] = {(cuuint64_t)2 * M, (cuuint64_t)M, (cuuint64_t)M, 8};
  cuuint64_t strides[3] = {(cuuint64_t)2 * M * 4, (cuuint64_t)2 * M * M * 4, (cuuint64_t)2 * M * M * M * 4};
  cuuint32_t box[4] = {zm::ROWF, zm::BY, 1, 4};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(in), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return QW_ECUDA;
  }
  s = smem_attr(zm::step3d_c64_tma_kernel, zm::SMEM_BYTES);
  if (s != QW_OK) return s;
  int dev = 0, nsm = 0;
  QW_CHECK_CUDA(cudaGetDevice(&dev));
  QW_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int resident = 2 * nsm;
  const int grid = nitems < resident ? nitems : resident;
  QW_CHECK_CUDA(cudaMemsetAsync(next_item, 0, sizeof(int), st));
  zm::step3d_c64_tma_kernel<<<grid, zm::NT, zm::SMEM_BYTES, st>>>(map, static_cast<const float2*>(in),
                                                                   static_cast<float2*>(out), M, items, nitems,
                                                                   make_coef32(3, n, m), err, next_item);
  QW_CHECK_LAUNCH("tma stencil launch");
  return QW_OK;
}

}  // namespace qw
