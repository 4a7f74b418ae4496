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

namespace qw {
namespace zm {

constexpr int TX = 64, TY = 4, NT = 128;  // tile (cells), threads: 32 x 4, two x-cells per thread
constexpr int BXC = TX + 4;               // box cells along x: [x0 - 2, x0 + TX + 2)
constexpr int BY = TY + 2;                // box rows: [y0 - 1, y0 + TY + 1)
constexpr int ROWF = 2 * BXC;             // floats per row
constexpr int CSTR = BY * ROWF;           // floats per component
constexpr int BUF_FLOATS = 4 * CSTR;
constexpr int BUF_BYTES = BUF_FLOATS * 4;
constexpr int NSLOT = 4;                  // ring depth per coset: two layer pairs in flight
constexpr int MAX_FIX = 3;                // periodic-image cells per thread per buffer
constexpr int SMEM_BYTES = 2 * NSLOT * BUF_BYTES + 2 * NSLOT * 8 + 128;  // + alignment slack
constexpr long long kSpinLimit = 1ll << 22;

static_assert(BUF_BYTES % 128 == 0, "TMA destinations must stay 128-byte aligned");
static_assert(ROWF <= 256 && BY <= 256, "TMA box extents");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false (and the error word set) if the copy never lands.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* err) {
  for (long long i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// acc += (A + i B) v for A, B in {-1, 0, 1}
template <int A, int B>
__device__ __forceinline__ void cmac(float2& acc, const float2& v) {
  if constexpr (A == 1) { acc.x += v.x; acc.y += v.y; }
  if constexpr (A == -1) { acc.x -= v.x; acc.y -= v.y; }
  if constexpr (B == 1) { acc.x -= v.y; acc.y += v.x; }
  if constexpr (B == -1) { acc.x += v.y; acc.y -= v.x; }
}

__device__ __forceinline__ float2 finish(const Coef32& c, float2 S, float2 o) {
  float rx = -c.m_lo * o.y;
  rx = fmaf(c.nq_lo, S.x, rx);
  rx = fmaf(-c.m_hi, o.y, rx);
  rx = fmaf(c.nq_hi, S.x, rx);
  float ry = c.m_lo * o.x;
  ry = fmaf(c.nq_lo, S.y, ry);
  ry = fmaf(c.m_hi, o.x, ry);
  ry = fmaf(c.nq_hi, S.y, ry);
  return make_float2(rx, ry);
}

struct Row3 {
  float2 lo, mid, hi;
};

// Row of one component: cells [lo, mid, hi] = tile-local x q0-1+C .. q0+1+C (q0 = 2 tx).
template <int C>
__device__ __forceinline__ Row3 srow(const float* row, int tx) {
  Row3 r;
  if constexpr (C == 0) {  // box columns q0+1, q0+2, q0+3
    const float2 a = *reinterpret_cast<const float2*>(row + 4 * tx + 2);
    const float4 b = *reinterpret_cast<const float4*>(row + 4 * tx + 4);
    r.lo = a;
    r.mid = make_float2(b.x, b.y);
    r.hi = make_float2(b.z, b.w);
  } else {                 // box columns q0+2, q0+3, q0+4
    const float4 a = *reinterpret_cast<const float4*>(row + 4 * tx + 4);
    const float2 b = *reinterpret_cast<const float2*>(row + 4 * tx + 8);
    r.lo = make_float2(a.x, a.y);
    r.mid = make_float2(a.z, a.w);
    r.hi = b;
  }
  return r;
}

template <int HY, int HZ>
__device__ __forceinline__ void pair(float2 (&S)[2][4], const Row3& a, const Row3& b, const Row3& cd) {
  constexpr int PP = HY * HZ, PM = -HY * HZ;
  if constexpr (HZ == 1) {
    cmac<1, -PP>(S[0][0], a.lo);  cmac<1, -HY>(S[0][0], b.lo);  cmac<-1, HY>(S[0][2], cd.lo);  cmac<1, -PP>(S[0][3], cd.lo);
    cmac<1, -PP>(S[1][0], a.mid); cmac<1, -HY>(S[1][0], b.mid); cmac<-1, HY>(S[1][2], cd.mid); cmac<1, -PP>(S[1][3], cd.mid);
    cmac<1, -PM>(S[0][0], a.mid); cmac<-1, -HY>(S[0][0], b.mid); cmac<1, HY>(S[0][2], cd.mid); cmac<1, -PM>(S[0][3], cd.mid);
    cmac<1, -PM>(S[1][0], a.hi);  cmac<-1, -HY>(S[1][0], b.hi);  cmac<1, HY>(S[1][2], cd.hi);  cmac<1, -PM>(S[1][3], cd.hi);
  } else {
    cmac<1, HY>(S[0][1], a.lo);  cmac<1, -PP>(S[0][1], b.lo);  cmac<1, -PP>(S[0][2], cd.lo);  cmac<-1, -HY>(S[0][3], cd.lo);
    cmac<1, HY>(S[1][1], a.mid); cmac<1, -PP>(S[1][1], b.mid); cmac<1, -PP>(S[1][2], cd.mid); cmac<-1, -HY>(S[1][3], cd.mid);
    cmac<-1, HY>(S[0][1], a.mid); cmac<1, -PM>(S[0][1], b.mid); cmac<1, -PM>(S[0][2], cd.mid); cmac<1, -HY>(S[0][3], cd.mid);
    cmac<-1, HY>(S[1][1], a.hi);  cmac<1, -PM>(S[1][1], b.hi);  cmac<1, -PM>(S[1][2], cd.hi);  cmac<1, -HY>(S[1][3], cd.hi);
  }
}

// Outputs of coset C at layer z for the thread's two cells.
//   lay_a: other coset at the h_z = +1 source layer, lay_b: at the h_z = -1 layer
//   own:   coset C at layer z (mass term)
template <int C>
__device__ __forceinline__ void compute(const float* lay_a, const float* lay_b, const float* own, float4* dst,
                                        int64_t v4, const Coef32& cf, int tx, int ty) {
  float2 S[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) S[j][q] = make_float2(0.f, 0.f);
  // box row of the h_y = +1 source: ty + C, of h_y = -1: ty + 1 + C
#pragma unroll
  for (int iy = 0; iy < 2; ++iy) {
    const int r = ty + C + iy;
    const float* base = lay_a + r * ROWF;
    Row3 a = srow<C>(base, tx), b = srow<C>(base + CSTR, tx), d = srow<C>(base + 3 * CSTR, tx);
    if (iy == 0) pair<+1, +1>(S, a, b, d); else pair<-1, +1>(S, a, b, d);
  }
#pragma unroll
  for (int iy = 0; iy < 2; ++iy) {
    const int r = ty + C + iy;
    const float* base = lay_b + r * ROWF;
    Row3 a = srow<C>(base, tx), b = srow<C>(base + CSTR, tx), c = srow<C>(base + 2 * CSTR, tx);
    if (iy == 0) pair<+1, -1>(S, a, b, c); else pair<-1, -1>(S, a, b, c);
  }
  const float* ob = own + (ty + 1) * ROWF + 4 * tx + 4;
  float4 o[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) o[q] = *reinterpret_cast<const float4*>(ob + q * CSTR);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 w = o[q ^ 2];
    const float2 r0 = finish(cf, S[0][q], make_float2(w.x, w.y));
    const float2 r1 = finish(cf, S[1][q], make_float2(w.z, w.w));
    dst[q * v4] = make_float4(r0.x, r0.y, r1.x, r1.y);
  }
}

struct Fix {
  int n;
  int soff[MAX_FIX];      // float offset inside a buffer
  int64_t goff[MAX_FIX];  // complex offset inside one coset (comp * vol + y * M + x)
};

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

    // Periodic images of this tile's out-of-range box cells.  The region is the
    // edge columns (all rows) plus the edge rows (remaining columns); the k-th
    // cell of that list, k = tid + i * NT, is this thread's i-th fix-up.
    Fix fx;
    {
      const bool xl = (x0 == 0), xr = (x0 + TX == M), yl = (y0 == 0), yr = (y0 + TY == M);
      const int nxo = 2 * (int)xl + 2 * (int)xr, nyo = (int)yl + (int)yr;
      const int nA = BY * nxo, nB = nyo * (BXC - nxo), per = nA + nB;
      const int total = 4 * per;
      if (total > MAX_FIX * NT) atomicExch(err, 2);  // cannot happen for TY < M
      fx.n = 0;
#pragma unroll
      for (int i = 0; i < MAX_FIX; ++i) {
        const int k = tid + i * NT;
        fx.soff[i] = 0;
        fx.goff[i] = 0;
        if (k < total) {
          const int cp = k / per, j = k % per;
          int r, q;
          if (j < nA) {
            r = j / nxo;
            const int oc = j % nxo;                      // 0, 1 -> left pair if xl, else right pair
            q = (xl && oc < 2) ? oc : TX + 2 + (oc & 1);
          } else {
            const int jj = j - nA, w = BXC - nxo;
            r = (yl && jj / w == 0) ? 0 : BY - 1;
            q = (jj % w) + (xl ? 2 : 0);
          }
          int x = x0 - 2 + q, y = y0 - 1 + r;
          x = x < 0 ? x + M : (x >= M ? x - M : x);
          y = y < 0 ? y + M : (y >= M ? y - M : y);
          fx.soff[i] = cp * CSTR + r * ROWF + 2 * q;
          fx.goff[i] = (int64_t)cp * vol + (int64_t)y * M + x;
          fx.n = i + 1;
        }
      }
    }

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
        compute<0>(c1m, c1z, c0z, d0, v4, cf, tx, ty);
        compute<1>(c0z, c0p, c1z, d1, v4, cf, tx, ty);
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

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static qw_status get_encoder() {
  if (g_encode) return QW_OK;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return QW_ECUDA;
  }
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return QW_OK;
}

bool tma_step_supported(const Geometry& g) {
  return g.dim == 3 && g.nx % zm::TX == 0 && g.nx >= zm::TX && g.nx <= 4096;
}

std::vector<int4> tma_item_table(const Geometry& g, int resident) {
  // Every tile's z-range is cut the same way: chunks of 64 layers while more
  // than a quarter of the box remains, then halving down to 8.  Items are
  // ordered chunk by chunk over all tiles, so the short chunks come last (the
  // tail of the dynamic schedule) and running CTAs work on neighbouring tiles
  // at similar depths (shared halo rows stay in L2).
  const int M = (int)g.nx;
  const int ntiles = (M / zm::TX) * (M / zm::TY);
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
  qw_status s = get_encoder();
  if (s != QW_OK) return s;
  const int M = (int)g.nx;
  CUtensorMap map;
  cuuint64_t dims[4] = {(cuuint64_t)2 * M, (cuuint64_t)M, (cuuint64_t)M, 8};
  cuuint64_t strides[3] = {(cuuint64_t)2 * M * 4, (cuuint64_t)2 * M * M * 4, (cuuint64_t)2 * M * M * M * 4};
  cuuint32_t box[4] = {zm::ROWF, zm::BY, 1, 4};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = g_encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(in), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return QW_ECUDA;
  }
  static bool attr_done = false;
  if (!attr_done) {
    QW_CHECK_CUDA(cudaFuncSetAttribute(zm::step3d_c64_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       zm::SMEM_BYTES));
    attr_done = true;
  }
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
