// Many independent walks of uneven size in one persistent launch (complex64).
//
// Work items are (walk, round, tile): round s < t_w of walk w applies the
// update rule (Eq. upd-rule, same per-site arithmetic as the plain kernels)
// to one tile of rows, from the walk's buffer s % 2 into (s + 1) % 2; for odd
// t_w a last round copies the result back into the caller's field.  Items are
// numbered in a fixed order and claimed through one atomic counter:
//   * walks are cut into groups whose two buffers fit in a share of L2;
//     groups follow one another, so a group's walks are evolved while cached;
//   * inside a group, rounds come in order and each round lists the tiles of
//     every walk still running (walks sorted by length, so that set is a prefix).
// Before working on round s of tile i of walk w a CTA waits (bounded) until the
// tiles within the stencil's reach of tile i (cyclically, the box is periodic)
// have finished round s-1: per-tile round counters, release/acquire (the lanes
// of warp 0 acquire the counters, then a CTA barrier orders the tile's loads).  That
// covers both the data tile i reads (written in round s-1) and the buffer it
// overwrites (read by its neighbours in round s-1), and lets consecutive rounds
// of a walk overlap as a wavefront instead of meeting at a barrier.  Every item
// waits only on items earlier in the order, and an item is only claimed by a
// running CTA, so the launch always makes progress.
// The launch (counter resets + kernel) is captured once into a CUDA graph and
// replayed by every qw_batch_run.
#include <cuda/atomic>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "qw_internal.cuh"
#include "qw_stencil_dev.cuh"

namespace qw {

struct BatchWalk {
  int dim;
  int ntiles;
  int reach;              // tiles on each side a tile depends on (cyclic)
  int64_t tile_base;      // first entry of this walk in the per-tile round counters
  int64_t nx;             // row length (N in 1D/2D, M = N/2 on the BCC lattice)
  int64_t ny;             // rows per plane layer (1 in 1D, N in 2D, M in 3D)
  int64_t rows;           // rows of one step (1, N, 2 M^2)
  int64_t rows_per_tile;
  int64_t t;
  int64_t rounds;         // t, plus one copy round when t is odd
  int64_t vol;            // complex values per component plane
  float2* buf[2];         // buf[0] = caller's field, buf[1] = partner
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

constexpr long long kBatchSpin = 1ll << 24;

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

__global__ void __launch_bounds__(256, 6) batch_kernel(const BatchWalk* __restrict__ walks,
                                                    const BatchGroup* __restrict__ groups,
                                                    const int64_t* __restrict__ group_item0, int ngroups,
                                                    const int64_t* __restrict__ tile_prefix,
                                                    const int64_t* __restrict__ round_prefix, int64_t total_items,
                                                    unsigned int* __restrict__ done, BatchCtl* __restrict__ ctl) {
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
    // wait for round s-1 of the tiles within reach, the lanes polling the tiles'
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
        const int ntiles = walks[wi].ntiles, reach = walks[wi].reach;
        const int64_t tbase = walks[wi].tile_base;
        const int span = 2 * reach + 1 >= ntiles ? ntiles : 2 * reach + 1;
        const int first = 2 * reach + 1 >= ntiles ? 0 : tile - reach;
        long long spins = 0;
        bool gave_up = false;
        for (int d = tid; d < span && !gave_up; d += 32) {
          int j = first + d;
          j = j < 0 ? j + ntiles : (j >= ntiles ? j - ntiles : j);
          cuda::atomic_ref<unsigned int, cuda::thread_scope_device> c(done[tbase + j]);
          while (c.load(cuda::memory_order_acquire) < (unsigned int)s) {
            if (++spins > kBatchSpin ||
                cuda::atomic_ref<int, cuda::thread_scope_device>(ctl->abort).load(cuda::memory_order_relaxed)) {
              cuda::atomic_ref<int, cuda::thread_scope_device>(ctl->abort).store(1, cuda::memory_order_relaxed);
              atomicExch(&ctl->err, 1);
              gave_up = true;
              break;
            }
            __nanosleep(64);
          }
        }
        if (gave_up) s_abort = 1;
      }
    }
    __syncthreads();
    if (s_abort) break;
    const int64_t s = s_round;
    const int tile = s_tile;
    const BatchWalk W = walks[s_walk];
    // claim the next item now (every thread read s_next before the barrier above): the
    // atomic's round trip overlaps this item's work, and the claimed item is started by
    // this CTA right after this one, so every claimed item still gets done
    if (tid == 0) s_next = (int64_t)atomicAdd(&ctl->next, 1ull);
    // ---- the tile's rows
    const int64_t r0 = (int64_t)tile * W.rows_per_tile;
    const int64_t r1 = min(W.rows, r0 + W.rows_per_tile);
    const int nx32 = (int)W.nx, ny32 = (int)W.ny;   // tiles and rows fit 32-bit indices
    const int nsite = (int)((r1 - r0) * W.nx);
    if (s < W.t) {
      // (buffers picked by selects: a dynamically indexed member array would put W in local memory)
      const float2* in = (s & 1) ? W.buf[1] : W.buf[0];
      float2* out = (s & 1) ? W.buf[0] : W.buf[1];
      // site k = tid + 256 i of the tile: (row, x) advanced by (256 / nx, 256 % nx) per
      // iteration, so no division per site; 32-bit indices (walks hold < 2^31 values)
      const int r0i = (int)r0;
      int kr = tid / nx32, x = tid - kr * nx32;
      const int dr = 256 / nx32, dx = 256 - dr * nx32;
      for (int k = tid; k < nsite; k += 256) {
        const int row = r0i + kr;
        if (W.dim == 1) {
          site_update_1d<float, false, int>(in, out, nx32, x, W.cf);
        } else if (W.dim == 2) {
          site_update_2d<float, false, int>(in, out, nx32, x, row, W.cf);
        } else {
          // rows interleave the cosets: row = 2 (z M + y) + c
          const int c = row & 1;
          const int zy = row >> 1;
          const int z = zy / ny32;
          site_update_3d<float, false, int>(in, out, nx32, c, z, zy - z * ny32, x, W.cf);
        }
        x += dx;
        kr += dr;
        if (x >= nx32) {
          x -= nx32;
          ++kr;
        }
      }
    } else {
      // copy round (odd t): the result sits in buf[1]
      const float2* src = W.buf[1];
      float2* dst = W.buf[0];
      const int s_comp = W.dim == 1 ? 2 : 4;
      for (int k = tid; k < nsite; k += blockDim.x) {
        const int kr = k / nx32;
        const int64_t row = r0 + kr, x = k - kr * nx32;
        int64_t base;
        if (W.dim == 3) {
          const int c = (int)(row & 1);
          base = (int64_t)c * 4 * W.vol + (row >> 1) * W.nx + x;
        } else {
          base = row * W.nx + x;
        }
        for (int q = 0; q < s_comp; ++q) dst[base + q * W.vol] = src[base + q * W.vol];
      }
    }
    __syncthreads();
    if (tid == 0) {
      cuda::atomic_ref<unsigned int, cuda::thread_scope_device>(done[W.tile_base + tile])
          .store((unsigned int)(s + 1), cuda::memory_order_release);
    }
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
  int64_t tile_sites = 4096;
  int64_t l2_budget = 48ll << 20;
  int grid = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // observables
  double* d_partials = nullptr;
  double* d_results = nullptr;
  double* h_results = nullptr;
};

namespace qw {

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

// Build the walk table, groups and prefix arrays for the current tile size and
// L2 budget, and upload them.
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
    if (grp.empty() || (acc + fb > b->l2_budget && !grp.back().empty())) {
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
  int64_t item0 = 0;
  int64_t ndone_acc = 0;
  for (auto& gw : grp) {
    // inside a group: longest walks first, so the walks alive at round s are a prefix
    std::stable_sort(gw.begin(), gw.end(), [&](int a, int c) { return b->desc[a].t > b->desc[c].t; });
    BatchGroup G;
    G.first = (int)walks.size();
    G.nw = (int)gw.size();
    G.tile_off = (int)tiles.size();
    G.round_off = (int)rounds.size();
    tiles.push_back(0);
    int64_t maxr = 0;
    std::vector<int64_t> wr;
    for (int i : gw) {
      const qw_walk& d = b->desc[i];
      Geometry g;
      make_geometry(d.dim, d.N, &g);
      BatchWalk W;
      W.dim = d.dim;
      W.nx = g.nx;
      W.ny = g.ny;
      W.rows = g.dim == 1 ? 1 : (g.dim == 2 ? g.ny : 2 * g.ny * g.nz);
      W.rows_per_tile = std::max<int64_t>(1, b->tile_sites / g.nx);
      W.ntiles = (int)((W.rows + W.rows_per_tile - 1) / W.rows_per_tile);
      // rows a site update reaches: 1 (2D), 2M + 3 (BCC rows interleave the cosets), 0 (1D: one row)
      const int64_t reach_rows = g.dim == 1 ? 0 : (g.dim == 2 ? 1 : 2 * g.nx + 3);
      // (+1 when the last tile is short: a cyclic neighbour window then needs one more tile)
      W.reach = (int)((reach_rows + W.rows_per_tile - 1) / W.rows_per_tile) + (W.rows % W.rows_per_tile ? 1 : 0);
      W.tile_base = ndone_acc;
      ndone_acc += W.ntiles;
      W.t = d.t;
      W.rounds = d.t + (d.t & 1);
      W.vol = g.vol;
      W.buf[0] = static_cast<float2*>(d.psi_dev);
      W.buf[1] = static_cast<float2*>(b->partners[i]);
      W.cf = make_coef32(d.dim, std::sqrt(1.0 - d.mass * d.mass), d.mass);
      walks.push_back(W);
      tiles.push_back(tiles.back() + W.ntiles);
      wr.push_back(W.rounds);
      maxr = std::max(maxr, W.rounds);
      b->order.push_back(i);
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
    // make round prefix relative to the group's first item
    item0 += G.nitems;
    groups.push_back(G);
  }
  // relative round prefixes: rounds[G.round_off + s] counts from the group's first item
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
  QW_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, 256, 0));
  QW_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device));
  b->grid = std::max(1, per_sm * nsm);
  return QW_OK;
}

static qw_status launch_batch(qw_batch_s* b, cudaStream_t s) {
  QW_CHECK_CUDA(cudaMemsetAsync(b->d_done, 0, std::max<int64_t>(1, b->ndone) * sizeof(unsigned int), s));
  QW_CHECK_CUDA(cudaMemsetAsync(b->d_ctl, 0, sizeof(BatchCtl), s));
  batch_kernel<<<b->grid, 256, 0, s>>>(b->d_walks, b->d_groups, b->d_group_item0, b->ngroups, b->d_tiles,
                                       b->d_rounds,
                                       b->total_items, b->d_done, b->d_ctl);
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
        w.t > 0x3fffffff) {
      set_error("qw_batch_create: walk %d has a bad dim/N/mass/t or a null field", i);
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

qw_status qw_batch_set_tiling(qw_batch b, int64_t tile_sites, int64_t l2_budget_bytes) {
  if (!b || tile_sites < 32 || tile_sites > (1 << 22) || l2_budget_bytes < (1 << 20)) {
    set_error("qw_batch_set_tiling: bad arguments (tile_sites in [32, 4M], budget >= 1 MiB)");
    return QW_EINVAL;
  }
  b->tile_sites = tile_sites;
  b->l2_budget = l2_budget_bytes;
  return build_schedule(b);
}

qw_status qw_batch_get_tiling(qw_batch b, int64_t* tile_sites, int64_t* l2_budget_bytes, int64_t* items) {
  if (!b) {
    set_error("qw_batch_get_tiling: null batch");
    return QW_EINVAL;
  }
  if (tile_sites) *tile_sites = b->tile_sites;
  if (l2_budget_bytes) *l2_budget_bytes = b->l2_budget;
  if (items) *items = b->total_items;
  return QW_OK;
}

qw_status qw_batch_run(qw_batch b, void* stream) {
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

qw_status qw_batch_autotune(qw_batch b, int64_t rounds_cap, void* stream, int64_t* best_tile, int64_t* best_budget,
                            double* best_rate) {
  if (!b || rounds_cap < 2) {
    set_error("qw_batch_autotune: null batch or rounds_cap < 2");
    return QW_EINVAL;
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
  const int64_t tiles[] = {1024, 2048, 4096, 8192, 16384};
  const int64_t budgets[] = {int64_t(24) << 20, int64_t(48) << 20, int64_t(96) << 20, int64_t(192) << 20,
                             int64_t(1) << 30, int64_t(16) << 30};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = -1.0;
  int64_t bt = b->tile_sites, bb = b->l2_budget;
  qw_status st = QW_OK;
  for (int64_t ts : tiles) {
    for (int64_t bu : budgets) {
      b->tile_sites = ts;
      b->l2_budget = bu;
      st = build_schedule(b);
      if (st != QW_OK) break;
      st = launch_batch(b, s);  // warm-up
      if (st != QW_OK) break;
      cudaEventRecord(e0, s);
      st = launch_batch(b, s);
      cudaEventRecord(e1, s);
      if (st != QW_OK) break;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double rate = (double)site_steps / (ms * 1e-3);
      if (rate > best) {
        best = rate;
        bt = ts;
        bb = bu;
      }
    }
    if (st != QW_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(pool);
  b->desc = real;
  b->tile_sites = bt;
  b->l2_budget = bb;
  qw_status st2 = build_schedule(b);
  if (st != QW_OK) return st;
  if (st2 != QW_OK) return st2;
  if (best_tile) *best_tile = bt;
  if (best_budget) *best_budget = bb;
  if (best_rate) *best_rate = best;
  return QW_OK;
}

qw_status qw_batch_observables(qw_batch b, qw_obs* out, void* stream) {
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
