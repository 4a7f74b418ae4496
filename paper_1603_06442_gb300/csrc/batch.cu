// Many independent walks of uneven size in one persistent launch (complex64).
//
// Every walk is cut into tiles: boxes of cells (x, y, z extents; on the BCC
// lattice a tile holds both cosets of its cells; the last tile of an axis may be
// shorter).  Work items are (walk, round, tile).  A round of walk w advances
// every tile of w by up to T_w steps of the update rule (Eq. upd-rule, the same
// per-site arithmetic as the plain kernels), from the walk's buffer r % 2 into
// (r + 1) % 2; when the number of stepping rounds is odd a last round copies
// the result back into the caller's field.  The fusion depth T_w is set per
// lattice dimension:
//   * T = 1: each cell is updated from global memory (the plain per-site update);
//   * T >= 2 (temporal fusion): the tile and a halo of H cells per side (H = T on
//     the chain and the square lattice, ceil(T/2) on the BCC lattice, where one
//     step reaches one cell of the other coset) are copied into shared memory by
//     cp.async; T steps run there over shrinking regions, and only the last one
//     is written to global memory: one read and one write of the field per T steps.
// Items are numbered in a fixed order and claimed through one atomic counter:
//   * walks are cut into groups whose two buffers fit in a share of L2;
//     groups follow one another, so a group's walks are evolved while cached;
//   * inside a group, rounds come in order and each round lists the tiles of
//     every walk still running (walks sorted by rounds, so that set is a prefix).
// Before round r of tile i of walk w a CTA waits (bounded) until every tile
// that meets tile i grown by H cells per axis (cyclically: the box is periodic)
// has finished round r - 1: per-tile round counters, release/acquire (the lanes
// of warp 0 acquire the counters, then a CTA barrier orders the tile's loads).
// That covers both the data the round reads (written in round r - 1) and the
// buffer it overwrites (read by its neighbours in round r - 1), and lets
// consecutive rounds of a walk overlap as a wavefront instead of meeting at a
// barrier.  Every item waits only on items earlier in the order, and an item is
// only claimed by a running CTA, so the launch always makes progress.
// The launch (counter resets + kernel) is captured once into a CUDA graph and
// replayed by every qw_batch_run.
#include <cuda/atomic>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <new>
#include <vector>

#include "qw_internal.cuh"
#include "qw_stencil_dev.cuh"

namespace qw {

struct BatchWalk {
  int dim;
  int depth;          // steps per round: 1 = per-site update from global memory, >= 2 = fused
  int halo;           // H: cells per side beyond the tile that one round depends on
  int ncos, ncomp;    // cosets (2 on the BCC lattice) and spinor components
  int n[3];           // cells per axis (nx, ny, nz)
  int ext[3];         // tile extents along x, y, z (cells)
  int nt[3];          // tiles per axis
  int ntiles;
  int vol;            // cells of one coset-component plane (walks hold < 2^31 values)
  int64_t tile_base;  // first entry of this walk in the per-tile round counters
  int64_t t;          // steps per run
  int64_t nstep;      // stepping rounds: ceil(t / depth)
  int64_t rounds;     // nstep, plus one copy round when nstep is odd
  float2* buf[2];     // buf[0] = caller's field, buf[1] = partner
  Coef32 cf;
};

struct BatchGroup {
  int first;        // first walk (index into the sorted walk table)
  int nw;
  int tile_off;     // offset of this group's tile prefix (nw + 1 entries)
  int round_off;    // offset of this group's round prefix (max rounds + 1 entries)
  int64_t nrounds;
  int64_t item0;    // first global item
  int64_t nitems;
};

struct BatchCtl {
  unsigned long long next;  // item counter
  int abort;                // set when a wait gave up
  int err;
};

// Fault injection for tests: the tile whose completions are never published (-1: none)
// and the number of polls after which a dependency wait gives up.
struct BatchDebug {
  int64_t stall_tile;
  long long spin_limit;
};

constexpr long long kBatchSpin = 1ll << 24;
constexpr int kBatchThreads = 256;   // plain (depth-1) launches
// plain launches: CTAs per SM the register budget is cut for (64 registers, no spills; 6 and 3
// CTAs, and cells taken two at a time, measured 2-15% slower on the uneven 256-walk mix)
constexpr int kBatchMinBlocks = 4;
constexpr int kFusedThreads = 256;   // launches with fused rounds (512 measured slower: 172 vs 232 G on the chain)

// Largest i in [0, n) with a[i] <= v (a ascending, a[0] <= v), searched by the 32 lanes
// of a warp together: each round cuts the range into 32 slices and keeps the last
// slice whose first element is <= v, so it takes log32(n) dependent loads instead of
// log2(n).  Every lane returns the same i.
__device__ __forceinline__ int64_t warp_upper_index(const int64_t* __restrict__ a, int64_t n, int64_t v, int lane) {
  int64_t lo = 0, len = n;  // a[lo] <= v; the answer lies in [lo, lo + len)
  while (len > 1) {
    const int64_t step = (len + 31) / 32, end = lo + len;
    const int64_t idx = lo + (int64_t)lane * step;
    const bool ok = idx < end && a[idx] <= v;
    const int c = __popc(__ballot_sync(0xffffffffu, ok));  // lanes 0 .. c-1 (a ascending)
    lo += (int64_t)(c - 1) * step;
    len = step < end - lo ? step : end - lo;
  }
  return lo;
}

// Calls f(x, y, z) for this thread's cells of the box [lo, hi) (per axis): cells
// tid, tid + NT, ... in x-fastest order, advanced without a division per cell.
template <int NT, typename F>
__device__ __forceinline__ void for_box(const int (&lo)[3], const int (&hi)[3], int tid, F&& f) {
  const int bx = hi[0] - lo[0], by = hi[1] - lo[1], bz = hi[2] - lo[2];
  const int n = bx * by * bz;
  if (tid >= n) return;
  int x = tid % bx, r = tid / bx;
  int y = r % by, z = r / by;
  const int dx = NT % bx, dr = NT / bx;
  const int dy = dr % by, dz = dr / by;
  for (int k = tid; k < n; k += NT) {
    f(lo[0] + x, lo[1] + y, lo[2] + z);
    x += dx;
    y += dy;
    z += dz;
    if (x >= bx) {
      x -= bx;
      ++y;
    }
    if (y >= by) {
      y -= by;
      ++z;
    }
  }
}

__device__ __forceinline__ int wrap_into(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// v mod n for v usually within one period of [0, n) (a halo never reaches further unless
// the walk is smaller than its halo): compares first, a division only otherwise.
__device__ __forceinline__ int wrap_near(int v, int n) {
  if (v < 0) v += n;
  else if (v >= n) v -= n;
  return (v < 0 || v >= n) ? wrap_into(v, n) : v;
}

// Region of coset c computed at step k of a fused round of `steps` steps, in the tile's
// local frame [0, e + 2H) per axis (axes >= dim: [0, 1)).  The last step covers the tile
// [H, H + e); going back one step, a BCC coset-0 cell needs coset 1 at m - 1 .. m and a
// coset-1 cell coset 0 at m .. m + 1 (the own cell of each too), so with j = steps - k:
// coset 0 [H - floor(j/2), H + e + ceil(j/2)), coset 1 [H - ceil(j/2), H + e + floor(j/2));
// on the chain and the square lattice every step reaches one cell: [H - j, H + e + j).
__device__ __forceinline__ void step_region(const BatchWalk& W, const int (&e)[3], int steps, int k, int c,
                                            int (&lo)[3], int (&hi)[3]) {
  const int j = steps - k, H = W.halo;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= W.dim) {
      lo[a] = 0;
      hi[a] = 1;
    } else if (W.dim == 3) {
      const int jl = c == 0 ? j / 2 : (j + 1) / 2, jh = c == 0 ? (j + 1) / 2 : j / 2;
      lo[a] = H - jl;
      hi[a] = H + e[a] + jh;
    } else {
      lo[a] = H - j;
      hi[a] = H + e[a] + j;
    }
  }
}

// cp.async of one 8-byte element into shared memory (all copies of a thread in flight).
__device__ __forceinline__ void cp_async8(float2* dst, const float2* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// One fused round of `steps` steps of tile (t0, t1, t2) of walk W: load the tile and its
// halo from `in` into shared buffer A, step there (A -> B -> A ...), write the last step
// to `out`.  Shared layout: [coset][component][z][y][x] with extents E = e + 2H per axis.
template <int NT>
__device__ __forceinline__ void fused_round(const BatchWalk& W, const int (&t3)[3], int steps, const float2* in, float2* out,
                            float2* smA, float2* smB) {
  const int tid = threadIdx.x;
  int s0[3], e[3], E[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    s0[a] = t3[a] * W.ext[a];
    e[a] = min(W.ext[a], W.n[a] - s0[a]);
    E[a] = a < W.dim ? e[a] + 2 * W.halo : 1;
  }
  const int H = W.halo;
  const int sy = E[0], sz = E[0] * E[1], P = sz * E[2];  // pitches, component stride
  const int nx = W.n[0], ny = W.n[1], nz = W.n[2];
  // ---- load: this thread's cells of the halo box (x fastest, so consecutive threads copy
  // consecutive x), each with every coset-component plane; periodic wrap per axis
  {
    const int lo3[3] = {0, 0, 0};
    const int planes = W.ncos * W.ncomp;
    for_box<NT>(lo3, E, tid, [&](int x, int y, int z) {
      const int gx = wrap_near(s0[0] - H + x, nx);
      const int gy = W.dim >= 2 ? wrap_near(s0[1] - H + y, ny) : 0;
      const int gz = W.dim >= 3 ? wrap_near(s0[2] - H + z, nz) : 0;
      const float2* src = in + ((int64_t)gz * ny + gy) * nx + gx;
      float2* dst = smA + z * sz + y * sy + x;
      for (int p = 0; p < planes; ++p) cp_async8(dst + p * P, src + (int64_t)p * W.vol);
    });
    cp_async_all();
  }
  __syncthreads();
  float2* cur = smA;
  float2* nxt = smB;
  for (int k = 1; k <= steps; ++k) {
    const bool last = k == steps;
    for (int c = 0; c < W.ncos; ++c) {
      int lo[3], hi[3];
      step_region(W, e, steps, k, c, lo, hi);
      for_box<NT>(lo, hi, tid, [&](int x, int y, int z) {
        const int i = z * sz + y * sy + x;  // 32-bit shared-memory offsets
        float2 r[4];
        if (W.dim == 1) {
          float2 r2[2];
          core_1d<false>(cur + i - 1, cur + i + 1, cur + i, P, r2, W.cf);
          r[0] = r2[0];
          r[1] = r2[1];
        } else if (W.dim == 2) {
          core_2d<false>(cur + i - 1, cur + i + 1, cur + i - sy, cur + i + sy, cur + i, P, r, W.cf);
        } else {
          core_3d<false>(cur + (1 - c) * 4 * P, sz, sy, z - 1 + c, z + c, y - 1 + c, y + c, x - 1 + c, x + c, P,
                         cur + c * 4 * P + i, r, W.cf);
        }
        if (last) {  // the tile's own cells: [H, H + e) maps to [s0, s0 + e), no wrap
          const int gx = s0[0] - H + x;
          const int gy = W.dim >= 2 ? s0[1] - H + y : 0;
          const int gz = W.dim >= 3 ? s0[2] - H + z : 0;
          float2* dst = out + (int64_t)c * W.ncomp * W.vol + ((int64_t)gz * ny + gy) * nx + gx;
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (q < W.ncomp) dst[(int64_t)q * W.vol] = r[q];
        } else {
          float2* dst = nxt + c * 4 * P + i;
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (q < W.ncomp) dst[q * P] = r[q];
        }
      });
    }
    if (!last) {
      __syncthreads();
      float2* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
  }
}

// U psi at site (x, y, z) of coset c: r[0..ncomp) and the index of its first output
// component (component q at i + q vol, vol the sites of one coset).
__device__ __forceinline__ int site_result(const BatchWalk& W, int c, int x, int y, int z, const float2* in,
                                           float2 (&r)[4]) {
  const int nx = W.n[0];
  if (W.dim == 1) {
    float2 r2[2];
    core_1d<false>(in + wrapm<int>(x - 1, nx), in + wrapm<int>(x + 1, nx), in + x, nx, r2, W.cf);
    r[0] = r2[0];
    r[1] = r2[1];
    return x;
  }
  if (W.dim == 2) {
    const int vol = nx * nx, i = y * nx + x;
    const int xm = wrapm<int>(x - 1, nx), xp = wrapm<int>(x + 1, nx);
    const int ym = wrapm<int>(y - 1, nx), yp = wrapm<int>(y + 1, nx);
    core_2d<false>(in + y * nx + xm, in + y * nx + xp, in + ym * nx + x, in + yp * nx + x, in + i, vol, r, W.cf);
    return i;
  }
  const int M = nx, plane = M * M, vol = plane * M;
  const int xa = wrapm<int>(x - 1 + c, M), xb = wrapm<int>(x + c, M);
  const int ya = wrapm<int>(y - 1 + c, M), yb = wrapm<int>(y + c, M);
  const int za = wrapm<int>(z - 1 + c, M), zb = wrapm<int>(z + c, M);
  const int i = z * plane + y * M + x;
  core_3d<false>(in + (1 - c) * 4 * vol, plane, M, za, zb, ya, yb, xa, xb, vol, in + c * 4 * vol + i, r, W.cf);
  return c * 4 * vol + i;
}

__device__ __forceinline__ void site_store(const BatchWalk& W, int i, const float2 (&r)[4], float2* out) {
  out[i] = r[0];
  out[i + W.vol] = r[1];
  if (W.ncomp == 4) {
    out[i + 2 * W.vol] = r[2];
    out[i + 3 * W.vol] = r[3];
  }
}

// The plain round of tile (t0, t1, t2): every cell of the tile (both cosets) updated once
// from global memory, or (copy round) copied from buf[1] to buf[0].
template <int NT>
__device__ __forceinline__ void plain_round(const BatchWalk& W, const int (&t3)[3], bool copy, const float2* in, float2* out) {
  int lo[3], hi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = t3[a] * W.ext[a];
    hi[a] = min(W.n[a], lo[a] + W.ext[a]);
  }
  const int nx = W.n[0], ny = W.n[1];
  for (int c = 0; c < W.ncos; ++c) {
    for_box<NT>(lo, hi, threadIdx.x, [&](int x, int y, int z) {
      if (copy) {
        const int64_t base = (int64_t)c * W.ncomp * W.vol + ((int64_t)z * ny + y) * nx + x;
        for (int q = 0; q < W.ncomp; ++q) out[base + (int64_t)q * W.vol] = in[base + (int64_t)q * W.vol];
      } else {
        float2 r[4];
        const int i = site_result(W, c, x, y, z, in, r);
        site_store(W, i, r, out);
      }
    });
  }
}

// FUSED = false: every walk has depth 1 (no shared memory, high occupancy);
// FUSED = true: walks of depth >= 2 run fused rounds in dynamic shared memory.
template <bool FUSED>
__global__ void __launch_bounds__(FUSED ? kFusedThreads : kBatchThreads, FUSED ? 3 : kBatchMinBlocks)
    batch_kernel(const BatchWalk* __restrict__ walks, const BatchGroup* __restrict__ groups,
                 const int64_t* __restrict__ group_item0, int ngroups, const int64_t* __restrict__ tile_prefix,
                 const int64_t* __restrict__ round_prefix, int64_t total_items, unsigned int* __restrict__ done,
                 BatchCtl* __restrict__ ctl, BatchDebug dbg) {
  extern __shared__ float2 smem_dyn[];
  __shared__ int64_t s_next, s_round;
  __shared__ int s_abort, s_walk, s_tile;
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_next = (int64_t)atomicAdd(&ctl->next, 1ull);
    s_abort = 0;
  }
  for (;;) {
    if (tid == 0 && cuda::atomic_ref<int, cuda::thread_scope_device>(ctl->abort).load(cuda::memory_order_relaxed))
      s_abort = 1;
    __syncthreads();
    const int64_t item = s_next;
    if (item >= total_items || s_abort) break;
    // ---- warp 0: decode (group, round, walk, tile) with warp-cooperative searches, then
    // wait for round s-1 of the tiles the round depends on, the lanes polling the tiles'
    // counters in parallel; the other warps wait at the barrier
    if (tid < 32) {
      const int g = (int)warp_upper_index(group_item0, ngroups, item, tid);
      const BatchGroup G = groups[g];
      const int64_t jj = item - G.item0;
      const int64_t* rp = round_prefix + G.round_off;
      const int64_t s = warp_upper_index(rp, G.nrounds + 1, jj, tid);
      const int64_t off = jj - rp[s];
      const int64_t* tp = tile_prefix + G.tile_off;
      const int wl = (int)warp_upper_index(tp, G.nw + 1, off, tid);
      const int tile = (int)(off - tp[wl]);
      const int wi = G.first + wl;
      if (tid == 0) {
        s_round = s;
        s_walk = wi;
        s_tile = tile;
      }
      if (s > 0) {
        const BatchWalk& W = walks[wi];
        // per axis: the cyclic range of tiles meeting [start - H, start + e + H)
        int first[3], cnt[3];
        const int t3[3] = {tile % W.nt[0], (tile / W.nt[0]) % W.nt[1], tile / (W.nt[0] * W.nt[1])};
        for (int a = 0; a < 3; ++a) {
          const int na = W.n[a], ea = W.ext[a], nta = W.nt[a];
          const int st = t3[a] * ea, e = min(ea, na - st);
          const int len = e + 2 * (a < W.dim ? W.halo : 0);
          if (len >= na) {
            first[a] = 0;
            cnt[a] = nta;
          } else {
            // cells lo .. lo + len - 1 (mod na): tiles lo / ea .. the end, then from tile 0 on
            // when the interval wraps past na - 1
            const int lo = wrap_into(st - (a < W.dim ? W.halo : 0), na), last = lo + len - 1;
            first[a] = lo / ea;
            const int c = last < na ? last / ea - first[a] + 1 : (nta - first[a]) + (last - na) / ea + 1;
            cnt[a] = min(c, nta);
          }
        }
        const int total = cnt[0] * cnt[1] * cnt[2];
        const long long limit = dbg.spin_limit;
        long long spins = 0;
        bool gave_up = false;
        for (int d = tid; d < total && !gave_up; d += 32) {
          const int i0 = d % cnt[0], r = d / cnt[0];
          const int i1 = r % cnt[1], i2 = r / cnt[1];
          const int j = (first[0] + i0) % W.nt[0] +
                        W.nt[0] * ((first[1] + i1) % W.nt[1] + W.nt[1] * ((first[2] + i2) % W.nt[2]));
          cuda::atomic_ref<unsigned int, cuda::thread_scope_device> c(done[W.tile_base + j]);
          while (c.load(cuda::memory_order_acquire) < (unsigned int)s) {
            if (++spins > limit ||
                cuda::atomic_ref<int, cuda::thread_scope_device>(ctl->abort).load(cuda::memory_order_relaxed)) {
              cuda::atomic_ref<int, cuda::thread_scope_device>(ctl->abort).store(1, cuda::memory_order_relaxed);
              atomicExch(&ctl->err, 1);
              gave_up = true;
              break;
            }
            __nanosleep(64);
          }
        }
        if (__any_sync(0xffffffffu, gave_up) && tid == 0) s_abort = 1;
      }
    }
    __syncthreads();
    if (s_abort) break;
    const int64_t s = s_round;
    const int tile = s_tile;
    // the walk's descriptor in registers: read through a reference, every field access in the
    // per-cell loops would be a global load that the field stores may alias
    const BatchWalk W = walks[s_walk];
    // claim the next item now (every thread read s_next before the barrier above): the
    // atomic's round trip overlaps this item's work, and the claimed item is started by
    // this CTA right after this one, so every claimed item still gets done
    if (tid == 0) s_next = (int64_t)atomicAdd(&ctl->next, 1ull);
    const int t3[3] = {tile % W.nt[0], (tile / W.nt[0]) % W.nt[1], tile / (W.nt[0] * W.nt[1])};
    // (buffers picked by selects: a dynamically indexed member array would go to local memory)
    float2* b0 = W.buf[0];
    float2* b1 = W.buf[1];
    if (s < W.nstep) {
      const float2* in = (s & 1) ? b1 : b0;
      float2* out = (s & 1) ? b0 : b1;
      const int steps = (int)min((int64_t)W.depth, W.t - s * W.depth);
      if (FUSED && W.depth > 1) {
        const int P = (W.ncos * W.ncomp) * (W.ext[0] + 2 * W.halo) * (W.dim >= 2 ? W.ext[1] + 2 * W.halo : 1) *
                      (W.dim >= 3 ? W.ext[2] + 2 * W.halo : 1);
        fused_round<FUSED ? kFusedThreads : kBatchThreads>(W, t3, steps, in, out, smem_dyn, smem_dyn + P);
      } else {
        plain_round<FUSED ? kFusedThreads : kBatchThreads>(W, t3, false, in, out);
      }
    } else {
      plain_round<FUSED ? kFusedThreads : kBatchThreads>(W, t3, true, b1, b0);  // copy round: the result sits in buf[1]
    }
    __syncthreads();
    if (tid == 0 && W.tile_base + tile != dbg.stall_tile) {
      __threadfence();
      cuda::atomic_ref<unsigned int, cuda::thread_scope_device>(done[W.tile_base + tile])
          .store((unsigned int)(s + 1), cuda::memory_order_release);
    }
  }
}

// qw_step's FUSED variant: `steps` updates of a whole field in one launch, one CTA per
// box tile (grid-stride), each a fused round from `in` to `out` (every tile reads only `in`,
// so the launch needs no dependency waits; successive launches ping-pong).
__global__ void __launch_bounds__(kFusedThreads, 3)
    fused_step_kernel(BatchWalk W, int steps, const float2* __restrict__ in, float2* __restrict__ out) {
  extern __shared__ float2 smem_dyn[];
  const int P = (W.ncos * W.ncomp) * (W.ext[0] + 2 * W.halo) * (W.dim >= 2 ? W.ext[1] + 2 * W.halo : 1) *
                (W.dim >= 3 ? W.ext[2] + 2 * W.halo : 1);
  for (int tile = blockIdx.x; tile < W.ntiles; tile += gridDim.x) {
    const int t3[3] = {tile % W.nt[0], (tile / W.nt[0]) % W.nt[1], tile / (W.nt[0] * W.nt[1])};
    fused_round<kFusedThreads>(W, t3, steps, in, out, smem_dyn, smem_dyn + P);
    __syncthreads();
  }
}

}  // namespace qw

using namespace qw;

struct qw_batch_s {
  int n = 0;
  int device = 0;
  std::vector<qw_walk> desc;      // caller's descriptors, original order
  std::vector<int> order;         // sorted position -> original index
  std::vector<void*> partners;    // per original walk
  BatchWalk* d_walks = nullptr;
  BatchGroup* d_groups = nullptr;
  int64_t* d_group_item0 = nullptr;  // first item of each group (warp search key)
  int64_t* d_tiles = nullptr;
  int64_t* d_rounds = nullptr;
  unsigned int* d_done = nullptr;
  int64_t ndone = 0;
  BatchCtl* d_ctl = nullptr;
  int ngroups = 0;
  int64_t total_items = 0;
  qw_batch_tiling tiling;
  bool fused = false;      // some walk has depth >= 2: the fused kernel runs the launch
  size_t smem = 0;         // its dynamic shared memory
  int grid = 0;
  BatchDebug dbg = {-1, kBatchSpin};
  int stall_walk = -1;     // caller's index of the walk whose first tile is stalled
  std::vector<int64_t> first_tile;  // per original walk: its first per-tile counter
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // observables
  double* d_partials = nullptr;
  double* d_results = nullptr;
  double* h_results = nullptr;
};

namespace qw {

// Defaults: what the autotuner picks for the 256-walk mix on GB300 (depth 1 on every lattice,
// 2048-site rows, one group); the boxes are those of fused rounds when a depth is raised.
static qw_batch_tiling default_tiling() {
  qw_batch_tiling t;
  t.tile_sites = 2048;
  t.l2_budget_bytes = int64_t(16) << 30;
  t.depth[0] = 1;
  t.depth[1] = 1;
  t.depth[2] = 1;
  const int box[3][3] = {{1024, 1, 1}, {32, 16, 1}, {8, 8, 4}};
  for (int d = 0; d < 3; ++d)
    for (int a = 0; a < 3; ++a) t.box[d][a] = box[d][a];
  return t;
}

static int halo_of(int dim, int depth) { return dim == 3 ? (depth + 1) / 2 : depth; }

// Shared memory of one fused round of a dim-dimensional walk with tile extents `box`
// (two buffers).
static size_t fused_smem(int dim, int depth, const int* box) {
  const int H = halo_of(dim, depth);
  size_t cells = 1;
  for (int a = 0; a < dim; ++a) cells *= (size_t)(box[a] + 2 * H);
  const int planes = dim == 1 ? 2 : (dim == 2 ? 4 : 8);  // cosets x components
  return 2 * cells * planes * sizeof(float2);
}

constexpr size_t kMaxBatchSmem = 227 * 1024;

static qw_status check_tiling(const qw_batch_tiling& t) {
  if (t.tile_sites < 32 || t.tile_sites > (1 << 22) || t.l2_budget_bytes < (1 << 20)) {
    set_error("qw_batch tiling: tile_sites in [32, 4M] and budget >= 1 MiB");
    return QW_EINVAL;
  }
  for (int d = 0; d < 3; ++d) {
    if (t.depth[d] < 1 || t.depth[d] > 4) {
      set_error("qw_batch tiling: fusion depth of dim %d is %d (1..4)", d + 1, t.depth[d]);
      return QW_EINVAL;
    }
    for (int a = 0; a <= d; ++a)
      if (t.box[d][a] < 1 || t.box[d][a] > 4096) {
        set_error("qw_batch tiling: box extent %d of dim %d out of range", t.box[d][a], d + 1);
        return QW_EINVAL;
      }
  }
  return QW_OK;
}

static void free_schedule(qw_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  if (b->d_walks) cudaFree(b->d_walks);
  if (b->d_groups) cudaFree(b->d_groups);
  if (b->d_group_item0) cudaFree(b->d_group_item0);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_rounds) cudaFree(b->d_rounds);
  if (b->d_done) cudaFree(b->d_done);
  b->d_walks = nullptr;
  b->d_groups = nullptr;
  b->d_group_item0 = nullptr;
  b->d_tiles = nullptr;
  b->d_rounds = nullptr;
  b->d_done = nullptr;
}

static int64_t field_bytes(const qw_walk& w) {
  Geometry g;
  make_geometry(w.dim, w.N, &g);
  return g.elems * 8;
}

// The walk's entry of the schedule under tiling t (tiles, depth, rounds).
static BatchWalk make_walk(const qw_walk& d, void* partner, const qw_batch_tiling& t) {
  Geometry g;
  make_geometry(d.dim, d.N, &g);
  BatchWalk W;
  W.dim = d.dim;
  W.depth = t.depth[d.dim - 1];
  W.ncos = g.ncoset;
  W.ncomp = g.s;
  W.n[0] = (int)g.nx;
  W.n[1] = (int)g.ny;
  W.n[2] = (int)g.nz;
  if (W.depth == 1) {
    // whole x rows (x segments on the chain), about tile_sites sites per tile
    W.halo = 1;
    if (d.dim == 1) {
      W.ext[0] = (int)std::min<int64_t>(g.nx, t.tile_sites);
      W.ext[1] = W.ext[2] = 1;
    } else {
      const int64_t rows = std::max<int64_t>(1, t.tile_sites / (g.nx * g.ncoset));
      W.ext[0] = (int)g.nx;
      W.ext[1] = (int)std::min<int64_t>(g.ny, rows);
      W.ext[2] = rows >= g.ny ? (int)std::min<int64_t>(g.nz, std::max<int64_t>(1, rows / g.ny)) : 1;
    }
  } else {
    W.halo = halo_of(d.dim, W.depth);
    for (int a = 0; a < 3; ++a) W.ext[a] = a < d.dim ? std::min(t.box[d.dim - 1][a], W.n[a]) : 1;
  }
  W.ntiles = 1;
  for (int a = 0; a < 3; ++a) {
    W.nt[a] = (W.n[a] + W.ext[a] - 1) / W.ext[a];
    W.ntiles *= W.nt[a];
  }
  W.vol = (int)g.vol;
  W.t = d.t;
  W.nstep = (d.t + W.depth - 1) / W.depth;
  W.rounds = W.nstep + (W.nstep & 1);
  W.buf[0] = static_cast<float2*>(d.psi_dev);
  W.buf[1] = static_cast<float2*>(partner);
  W.cf = make_coef32(d.dim, std::sqrt(1.0 - d.mass * d.mass), d.mass);
  W.tile_base = 0;
  return W;
}

bool fused_step_supported(const Geometry& g, qw_dtype dt, int depth, const int* box) {
  if (dt != QW_C64 || depth < 2 || depth > 4 || g.elems >= (int64_t(1) << 31)) return false;
  int ext[3];
  for (int a = 0; a < 3; ++a) {
    if (a < g.dim && box[a] < 1) return false;
    ext[a] = a < g.dim ? (int)std::min<int64_t>(box[a], a == 0 ? g.nx : (a == 1 ? g.ny : g.nz)) : 1;
  }
  return fused_smem(g.dim, depth, ext) <= kMaxBatchSmem;
}

qw_status launch_step_fused(const Geometry& g, int depth, const int* box, int steps, double n, double m,
                            const void* in, void* out, cudaStream_t st) {
  if (!fused_step_supported(g, QW_C64, depth, box) || steps < 1 || steps > depth) {
    set_error("fused stencil: unsupported geometry, depth %d, box or step count %d", depth, steps);
    return QW_EINVAL;
  }
  qw_walk d;
  d.dim = g.dim;
  d.N = g.N;
  d.mass = m;
  d.t = steps;
  d.psi_dev = const_cast<void*>(in);
  qw_batch_tiling t = default_tiling();
  t.depth[g.dim - 1] = depth;
  for (int a = 0; a < 3; ++a) t.box[g.dim - 1][a] = box[a];
  BatchWalk W = make_walk(d, out, t);
  W.cf = make_coef32(g.dim, n, m);
  const size_t smem = fused_smem(W.dim, W.depth, W.ext);
  qw_status sa = smem_attr(fused_step_kernel, (int)smem);
  if (sa != QW_OK) return sa;
  int dev = 0, nsm = 0, per_sm = 0;
  QW_CHECK_CUDA(cudaGetDevice(&dev));
  QW_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  QW_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_step_kernel, kFusedThreads, smem));
  const int grid = (int)std::min<int64_t>(W.ntiles, (int64_t)std::max(1, per_sm) * nsm);
  fused_step_kernel<<<grid, kFusedThreads, smem, st>>>(W, steps, static_cast<const float2*>(in),
                                                       static_cast<float2*>(out));
  QW_CHECK_LAUNCH("fused stencil launch");
  return QW_OK;
}

// Build the walk table, groups and prefix arrays for the current tiling, and upload them.
static qw_status build_schedule(qw_batch_s* b) {
  free_schedule(b);
  const int n = b->n;
  // sort by footprint (small walks first: they share L2 best), ties by length
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return field_bytes(b->desc[a]) < field_bytes(b->desc[c]); });
  // groups: consecutive walks whose two buffers fit the L2 budget
  std::vector<std::vector<int>> grp;
  int64_t acc = 0;
  for (int i : idx) {
    const int64_t fb = 2 * field_bytes(b->desc[i]);
    if (grp.empty() || (acc + fb > b->tiling.l2_budget_bytes && !grp.back().empty())) {
      grp.emplace_back();
      acc = 0;
    }
    grp.back().push_back(i);
    acc += fb;
  }
  std::vector<BatchWalk> walks;
  std::vector<BatchGroup> groups;
  std::vector<int64_t> tiles, rounds;
  b->order.clear();
  b->first_tile.assign(n, 0);
  b->fused = false;
  b->smem = 0;
  int64_t item0 = 0;
  int64_t ndone_acc = 0;
  for (auto& gw : grp) {
    std::vector<BatchWalk> gwalks;
    for (int i : gw) gwalks.push_back(make_walk(b->desc[i], b->partners[i], b->tiling));
    // inside a group: most rounds first, so the walks alive at round s are a prefix
    std::vector<int> ord(gw.size());
    for (size_t k = 0; k < gw.size(); ++k) ord[k] = (int)k;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) { return gwalks[a].rounds > gwalks[c].rounds; });
    BatchGroup G;
    G.first = (int)walks.size();
    G.nw = (int)gw.size();
    G.tile_off = (int)tiles.size();
    G.round_off = (int)rounds.size();
    tiles.push_back(0);
    int64_t maxr = 0;
    std::vector<int64_t> wr;
    for (int k : ord) {
      BatchWalk W = gwalks[k];
      W.tile_base = ndone_acc;
      b->first_tile[gw[k]] = ndone_acc;
      ndone_acc += W.ntiles;
      if (W.depth > 1) {
        // the box clipped to the walk: a box larger than a small walk costs nothing extra
        const size_t need = fused_smem(W.dim, W.depth, W.ext);
        if (need > kMaxBatchSmem) {
          set_error("qw_batch tiling: a dim-%d walk's tile with depth %d needs %zu bytes of shared memory (max %zu)",
                    W.dim, W.depth, need, kMaxBatchSmem);
          return QW_EINVAL;
        }
        b->fused = true;
        b->smem = std::max(b->smem, need);
      }
      walks.push_back(W);
      tiles.push_back(tiles.back() + W.ntiles);
      wr.push_back(W.rounds);
      maxr = std::max(maxr, W.rounds);
      b->order.push_back(gw[k]);
    }
    // round prefix: items of round s = tiles of the walks with rounds > s (a prefix)
    rounds.push_back(0);
    size_t alive = gw.size();
    for (int64_t s = 0; s < maxr; ++s) {
      while (alive > 0 && wr[alive - 1] <= s) --alive;
      rounds.push_back(rounds.back() + (tiles[G.tile_off + alive] - tiles[G.tile_off]));
    }
    G.nrounds = maxr;
    G.item0 = item0;
    G.nitems = rounds.back() - rounds[G.round_off];
    item0 += G.nitems;
    groups.push_back(G);
  }
  // relative prefixes: rounds[G.round_off + s] and tiles[G.tile_off + w] count from the group's start
  for (auto& G : groups) {
    const int64_t base = rounds[G.round_off];
    for (int64_t s = 0; s <= G.nrounds; ++s) rounds[G.round_off + s] -= base;
  }
  for (auto& G : groups) {
    const int64_t base = tiles[G.tile_off];
    for (int w = 0; w <= G.nw; ++w) tiles[G.tile_off + w] -= base;
  }
  b->ngroups = (int)groups.size();
  b->total_items = item0;
  b->dbg.stall_tile = b->stall_walk >= 0 ? b->first_tile[b->stall_walk] : -1;
  QW_CHECK_CUDA(cudaMalloc(&b->d_walks, walks.size() * sizeof(BatchWalk)));
  QW_CHECK_CUDA(cudaMalloc(&b->d_groups, groups.size() * sizeof(BatchGroup)));
  QW_CHECK_CUDA(cudaMalloc(&b->d_tiles, tiles.size() * sizeof(int64_t)));
  QW_CHECK_CUDA(cudaMalloc(&b->d_rounds, rounds.size() * sizeof(int64_t)));
  b->ndone = ndone_acc;
  QW_CHECK_CUDA(cudaMalloc(&b->d_done, std::max<int64_t>(1, ndone_acc) * sizeof(unsigned int)));
  QW_CHECK_CUDA(cudaMemcpy(b->d_walks, walks.data(), walks.size() * sizeof(BatchWalk), cudaMemcpyHostToDevice));
  QW_CHECK_CUDA(cudaMemcpy(b->d_groups, groups.data(), groups.size() * sizeof(BatchGroup), cudaMemcpyHostToDevice));
  std::vector<int64_t> gi0(groups.size());
  for (size_t i = 0; i < groups.size(); ++i) gi0[i] = groups[i].item0;
  QW_CHECK_CUDA(cudaMalloc(&b->d_group_item0, gi0.size() * sizeof(int64_t)));
  QW_CHECK_CUDA(cudaMemcpy(b->d_group_item0, gi0.data(), gi0.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  QW_CHECK_CUDA(cudaMemcpy(b->d_tiles, tiles.data(), tiles.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  QW_CHECK_CUDA(cudaMemcpy(b->d_rounds, rounds.data(), rounds.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  int per_sm = 0, nsm = 0;
  if (b->fused) {
    qw_status sa = smem_attr(batch_kernel<true>, (int)b->smem);
    if (sa != QW_OK) return sa;
    QW_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<true>, kFusedThreads, b->smem));
  } else {
    QW_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<false>, kBatchThreads, 0));
  }
  QW_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device));
  b->grid = std::max(1, per_sm * nsm);
  return QW_OK;
}

static qw_status launch_batch(qw_batch_s* b, cudaStream_t s) {
  if (debug_poison())  // every round writes its tile of the partner before any round reads it
    for (int i = 0; i < b->n; ++i)
      QW_CHECK_CUDA(cudaMemsetAsync(b->partners[i], kPoisonByte, field_bytes(b->desc[i]), s));
  QW_CHECK_CUDA(cudaMemsetAsync(b->d_done, 0, std::max<int64_t>(1, b->ndone) * sizeof(unsigned int), s));
  QW_CHECK_CUDA(cudaMemsetAsync(b->d_ctl, 0, sizeof(BatchCtl), s));
  if (b->fused)
    batch_kernel<true><<<b->grid, kFusedThreads, b->smem, s>>>(b->d_walks, b->d_groups, b->d_group_item0,
                                                               b->ngroups, b->d_tiles, b->d_rounds, b->total_items,
                                                               b->d_done, b->d_ctl, b->dbg);
  else
    batch_kernel<false><<<b->grid, kBatchThreads, 0, s>>>(b->d_walks, b->d_groups, b->d_group_item0, b->ngroups,
                                                          b->d_tiles, b->d_rounds, b->total_items, b->d_done,
                                                          b->d_ctl, b->dbg);
  QW_CHECK_LAUNCH("batch kernel launch");
  return QW_OK;
}

}  // namespace qw

extern "C" {

qw_status qw_batch_create(const qw_walk* walks, int n, qw_batch* out) {
  if (!out || !walks || n <= 0) {
    set_error("qw_batch_create: null argument or n <= 0");
    return QW_EINVAL;
  }
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    Geometry g;
    const qw_walk& w = walks[i];
    if (!make_geometry(w.dim, w.N, &g) || !(w.mass >= 0.0 && w.mass <= 1.0) || w.t < 0 || !w.psi_dev ||
        w.t > 0x3fffffff || g.elems >= (int64_t(1) << 31)) {
      set_error("qw_batch_create: walk %d has a bad dim/N/mass/t, more than 2^31 values or a null field", i);
      return QW_EINVAL;
    }
  }
  qw_batch_s* b = new (std::nothrow) qw_batch_s();
  if (!b) {
    set_error("qw_batch_create: host allocation failed");
    return QW_ENOMEM;
  }
  b->n = n;
  b->desc.assign(walks, walks + n);
  b->partners.assign(n, nullptr);
  b->tiling = default_tiling();
  qw_status st = QW_OK;
  cudaError_t e = cudaGetDevice(&b->device);
  for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaMalloc(&b->partners[i], field_bytes(walks[i]));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_ctl, sizeof(BatchCtl));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_partials, sizeof(double) * 4 * kObsBlocks);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_results, sizeof(double) * 4 * n);
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_results, sizeof(double) * 4 * n);
  if (e == cudaSuccess) e = cudaMemset(b->d_ctl, 0, sizeof(BatchCtl));
  if (e != cudaSuccess) {
    st = cuda_fail(e, "qw_batch_create: allocation");
    qw_batch_destroy(b);
    return st;
  }
  st = build_schedule(b);
  if (st != QW_OK) {
    qw_batch_destroy(b);
    return st;
  }
  *out = b;
  return QW_OK;
}

qw_status qw_batch_destroy(qw_batch b) {
  if (!b) return QW_OK;
  cudaDeviceSynchronize();
  free_schedule(b);
  for (void* p : b->partners)
    if (p) cudaFree(p);
  if (b->d_ctl) cudaFree(b->d_ctl);
  if (b->d_partials) cudaFree(b->d_partials);
  if (b->d_results) cudaFree(b->d_results);
  if (b->h_results) cudaFreeHost(b->h_results);
  delete b;
  return QW_OK;
}

qw_status qw_batch_set_tiling(qw_batch b, const qw_batch_tiling* tiling) {
  if (!b || !tiling) {
    set_error("qw_batch_set_tiling: null argument");
    return QW_EINVAL;
  }
  qw_status st = check_tiling(*tiling);
  if (st != QW_OK) return st;
  b->tiling = *tiling;
  return build_schedule(b);
}

qw_status qw_batch_get_tiling(qw_batch b, qw_batch_tiling* tiling, int64_t* items) {
  if (!b) {
    set_error("qw_batch_get_tiling: null batch");
    return QW_EINVAL;
  }
  if (tiling) *tiling = b->tiling;
  if (items) *items = b->total_items;
  return QW_OK;
}

qw_status qw_batch_debug_stall(qw_batch b, int walk, int64_t spin_limit) {
  if (!b || walk >= b->n || (walk >= 0 && spin_limit < 1)) {
    set_error("qw_batch_debug_stall: null batch, walk index out of range or spin_limit < 1");
    return QW_EINVAL;
  }
  b->stall_walk = walk < 0 ? -1 : walk;
  b->dbg.spin_limit = walk < 0 ? kBatchSpin : spin_limit;
  return build_schedule(b);  // drops the captured graph: its kernel arguments change
}

qw_status qw_batch_run(qw_batch b, void* stream) {
  NvtxRange nvtx_range("qw_batch_run");
  if (!b) {
    set_error("qw_batch_run: null batch");
    return QW_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!b->exec) {
    // capture the launch once on a private stream, then replay it
    cudaStream_t cap;
    QW_CHECK_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    QW_CHECK_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    qw_status st = launch_batch(b, cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    if (st != QW_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "qw_batch_run: capture");
    b->graph = graph;
    QW_CHECK_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
  }
  QW_CHECK_CUDA(cudaGraphLaunch(b->exec, s));
  return QW_OK;
}

qw_status qw_batch_sync(qw_batch b, void* stream) {
  if (!b) {
    set_error("qw_batch_sync: null batch");
    return QW_EINVAL;
  }
  BatchCtl ctl;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  QW_CHECK_CUDA(cudaMemcpyAsync(&ctl, b->d_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
  QW_CHECK_CUDA(cudaStreamSynchronize(s));
  if (ctl.err) {
    set_error("qw_batch_run: a bounded dependency wait gave up; walk results are invalid");
    return QW_ETIMEOUT;
  }
  return QW_OK;
}

qw_status qw_batch_autotune(qw_batch b, int64_t rounds_cap, void* stream, qw_batch_tiling* best_tiling,
                            double* best_rate) {
  NvtxRange nvtx_range("qw_batch_autotune");
  if (!b || rounds_cap < 2) {
    set_error("qw_batch_autotune: null batch or rounds_cap < 2");
    return QW_EINVAL;
  }
  if (b->stall_walk >= 0) {
    set_error("qw_batch_autotune: a stall is injected (qw_batch_debug_stall); clear it first");
    return QW_EINVAL;
  }
  // the cache key: the walks' (dim, N, t) in the caller's order (FNV-1a) and the tuning length
  uint64_t h = 1469598103934665603ull;
  auto mix = [&h](uint64_t v) {
    for (int k = 0; k < 8; ++k) {
      h ^= (v >> (8 * k)) & 0xff;
      h *= 1099511628211ull;
    }
  };
  for (const qw_walk& w : b->desc) {
    mix((uint64_t)w.dim);
    mix((uint64_t)w.N);
    mix((uint64_t)w.t);
  }
  char problem[96];
  std::snprintf(problem, sizeof(problem), "walks=%d mix=%016llx cap=%lld", b->n, (unsigned long long)h,
                (long long)rounds_cap);
  std::vector<double> cached;
  if (autotune_cache_get("batch", problem, &cached) && cached.size() == 15) {
    qw_batch_tiling t;
    t.tile_sites = (int64_t)cached[0];
    t.l2_budget_bytes = (int64_t)cached[1];
    for (int d = 0; d < 3; ++d) {
      t.depth[d] = (int)cached[2 + d];
      for (int a = 0; a < 3; ++a) t.box[d][a] = (int)cached[5 + 3 * d + a];
    }
    if (check_tiling(t) == QW_OK) {  // the measured choice of an earlier run on this GPU model
      b->tiling = t;
      qw_status st = build_schedule(b);
      if (st != QW_OK) return st;
      if (best_tiling) *best_tiling = t;
      if (best_rate) *best_rate = cached[14];
      return QW_OK;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // stand-in fields of the same sizes (the walks' own fields are left untouched)
  std::vector<qw_walk> real = b->desc;
  int64_t total = 0;
  for (auto& w : real) total += field_bytes(w);
  void* pool = nullptr;
  QW_CHECK_CUDA(cudaMalloc(&pool, total));
  QW_CHECK_CUDA(cudaMemsetAsync(pool, 0, total, s));
  int64_t off = 0;
  int64_t site_steps = 0;
  int64_t tmax = 1;
  for (auto& w : b->desc) tmax = std::max<int64_t>(tmax, w.t);
  for (auto& w : b->desc) {
    w.psi_dev = static_cast<char*>(pool) + off;
    off += field_bytes(w);
    // step counts scaled so the longest walk runs rounds_cap steps: the tuning run keeps the
    // mix's shape, the tail of the longest walks included (capping every walk would drop it)
    if (tmax > rounds_cap) w.t = std::max<int64_t>(1, (w.t * rounds_cap + tmax - 1) / tmax);
    Geometry g;
    make_geometry(w.dim, w.N, &g);
    site_steps += g.sites * w.t;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const qw_batch_tiling saved = b->tiling;
  qw_batch_tiling best = saved;
  double best_r = -1.0;
  qw_status st = QW_OK;
  auto measure = [&](const qw_batch_tiling& t) -> qw_status {
    if (check_tiling(t) != QW_OK) return QW_OK;  // not a candidate
    b->tiling = t;
    qw_status r = build_schedule(b);
    if (r == QW_EINVAL) return QW_OK;  // a tile of this mix does not fit shared memory
    if (r != QW_OK) return r;
    if ((r = launch_batch(b, s)) != QW_OK) return r;  // warm-up
    cudaEventRecord(e0, s);
    if ((r = launch_batch(b, s)) != QW_OK) return r;
    cudaEventRecord(e1, s);
    QW_CHECK_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double rate = (double)site_steps / (ms * 1e-3);
    if (rate > best_r) {
      best_r = rate;
      best = t;
    }
    return QW_OK;
  };
  // stage 1: one step per round, whole-row tiles of each size
  const int64_t tiles[] = {1024, 2048, 4096, 8192};
  qw_batch_tiling t = default_tiling();
  t.depth[0] = t.depth[1] = t.depth[2] = 1;
  for (int64_t ts : tiles) {
    if (st != QW_OK) break;
    t.tile_sites = ts;
    st = measure(t);
  }
  // stage 2: fused rounds, fusion depth and tile box per lattice (depth-1 walks keep the
  // best row tile of stage 1)
  const int depth2[] = {2, 4};
  const int depth3[] = {1, 2};
  const int box2[][3] = {{32, 16, 1}, {64, 8, 1}, {32, 32, 1}, {64, 16, 1}};
  const int box3[][3] = {{8, 8, 4}, {8, 8, 6}, {16, 8, 4}, {8, 8, 8}};
  const int64_t best_rows = best.tile_sites;
  for (int d2 : depth2)
    for (const auto& bx2 : box2)
      for (int d3 : depth3)
        for (int k3 = 0; k3 < (d3 == 1 ? 1 : 4) && st == QW_OK; ++k3) {
          t = default_tiling();
          t.tile_sites = best_rows;
          t.depth[0] = t.depth[1] = d2;
          t.depth[2] = d3;
          for (int a = 0; a < 3; ++a) {
            t.box[1][a] = bx2[a];
            t.box[2][a] = box3[k3][a];
          }
          st = measure(t);
        }
  // stage 3: the group budget for the best tiling (small budgets keep a group in L2)
  const int64_t budgets[] = {int64_t(48) << 20, int64_t(96) << 20, int64_t(192) << 20, int64_t(1) << 30};
  const qw_batch_tiling stage2 = best;
  for (int64_t bu : budgets) {
    if (st != QW_OK) break;
    t = stage2;
    t.l2_budget_bytes = bu;
    st = measure(t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(pool);
  b->desc = real;
  b->tiling = st == QW_OK ? best : saved;
  qw_status st2 = build_schedule(b);
  if (st != QW_OK) return st;
  if (st2 != QW_OK) return st2;
  std::vector<double> v = {(double)best.tile_sites, (double)best.l2_budget_bytes};
  for (int d = 0; d < 3; ++d) v.push_back(best.depth[d]);
  for (int d = 0; d < 3; ++d)
    for (int a = 0; a < 3; ++a) v.push_back(best.box[d][a]);
  v.push_back(best_r);
  autotune_cache_put("batch", problem, v);
  if (best_tiling) *best_tiling = best;
  if (best_rate) *best_rate = best_r;
  return QW_OK;
}

qw_status qw_batch_observables(qw_batch b, qw_obs* out, void* stream) {
  NvtxRange nvtx_range("qw_batch_observables");
  if (!b || !out) {
    set_error("qw_batch_observables: null argument");
    return QW_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < b->n; ++i) {
    Geometry g;
    make_geometry(b->desc[i].dim, b->desc[i].N, &g);
    qw_status st = launch_position_moments(g, QW_C64, b->desc[i].psi_dev, b->d_partials, b->d_results + 4 * i, s);
    if (st != QW_OK) return st;
  }
  QW_CHECK_CUDA(cudaMemcpyAsync(b->h_results, b->d_results, sizeof(double) * 4 * b->n, cudaMemcpyDeviceToHost, s));
  qw_status st = qw_batch_sync(b, stream);
  if (st != QW_OK) return st;
  for (int i = 0; i < b->n; ++i) {
    const double* r = b->h_results + 4 * i;
    out[i].norm = r[0];
    for (int j = 0; j < 3; ++j) out[i].x_mean[j] = (j < b->desc[i].dim && r[0] > 0) ? r[1 + j] / r[0] : 0.0;
    out[i].w_particle = NAN;
    out[i].w_antiparticle = NAN;
  }
  return QW_OK;
}

}  // extern "C"
