// C ABI entry points: errors, plans, the stepping driver and observables.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <tuple>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "qw_internal.cuh"

namespace qw {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

qw_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  return e == cudaErrorMemoryAllocation ? QW_ENOMEM : QW_ECUDA;
}

qw_status smem_attr_once(const void* func, int bytes) {
  // the attribute is an upper bound: it is only ever raised, to the largest size requested
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> limit;
  int dev = 0;
  QW_CHECK_CUDA(cudaGetDevice(&dev));
  const auto key = std::make_pair(func, dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = limit.find(key);
  if (it != limit.end() && it->second >= bytes) return QW_OK;
  QW_CHECK_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  limit[key] = bytes;
  return QW_OK;
}

int resident_blocks_once(const void* func, int threads, int smem) {
  // blocks of func resident on the whole device (per-SM occupancy x SMs), per device
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, int, int>, int> known;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  const auto key = std::make_tuple(func, dev, threads, smem);
  std::lock_guard<std::mutex> lock(mu);
  auto it = known.find(key);
  if (it != known.end()) return it->second;
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, smem) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return known[key] = per_sm * sms;
}

static std::atomic<bool> g_poison{false};
bool debug_poison() { return g_poison.load(std::memory_order_relaxed); }

static std::mutex g_cache_mu;
static std::string g_cache_path;  // empty: no autotune cache

// "<kind> <GPU model> <problem>" (spaces in the model name become '_')
static std::string cache_key(const char* kind, const char* problem) {
  int dev = 0;
  cudaDeviceProp prop;
  std::string name = "unknown-gpu";
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
  for (char& c : name)
    if (c == ' ') c = '_';
  return std::string(kind) + " " + name + " " + problem;
}

bool autotune_cache_get(const char* kind, const char* problem, std::vector<double>* values) {
  std::lock_guard<std::mutex> lock(g_cache_mu);
  if (g_cache_path.empty()) return false;
  FILE* f = std::fopen(g_cache_path.c_str(), "r");
  if (!f) return false;
  const std::string key = cache_key(kind, problem) + " |";
  char line[1024];
  bool found = false;
  while (std::fgets(line, sizeof(line), f)) {
    if (std::strncmp(line, key.c_str(), key.size()) != 0) continue;
    std::vector<double> v;
    const char* p = line + key.size();
    char* end = nullptr;
    for (double x = std::strtod(p, &end); end != p; x = std::strtod(p, &end)) {
      v.push_back(x);
      p = end;
    }
    *values = v;  // the last matching line wins
    found = true;
  }
  std::fclose(f);
  return found;
}

void autotune_cache_put(const char* kind, const char* problem, const std::vector<double>& values) {
  std::lock_guard<std::mutex> lock(g_cache_mu);
  if (g_cache_path.empty()) return;
  FILE* f = std::fopen(g_cache_path.c_str(), "a");
  if (!f) return;
  std::string line = cache_key(kind, problem) + " |";
  char buf[64];
  for (double x : values) {
    std::snprintf(buf, sizeof(buf), " %.17g", x);
    line += buf;
  }
  std::fprintf(f, "%s\n", line.c_str());
  std::fclose(f);
}

bool make_geometry(int dim, int64_t N, Geometry* g) {
  if (dim < 1 || dim > 3 || N < 2) return false;
  g->dim = dim;
  g->N = N;
  g->s = (dim == 1) ? 2 : 4;
  if (dim == 1) {
    g->ncoset = 1;
    g->nx = N;
    g->ny = g->nz = 1;
  } else if (dim == 2) {
    g->ncoset = 1;
    g->nx = g->ny = N;
    g->nz = 1;
  } else {
    if (N % 2 != 0) return false;
    g->ncoset = 2;
    g->nx = g->ny = g->nz = N / 2;
  }
  g->vol = g->nx * g->ny * g->nz;
  g->elems = (int64_t)g->ncoset * g->s * g->vol;
  g->sites = (int64_t)g->ncoset * g->vol;
  return true;
}

static int default_stencil(const qw_plan_s* p) {
  // measured on GB300: BCC N = 512, the fused two-step kernel (one HBM pass per two steps,
  // shared-memory bound) ahead of the one-step TMA kernel (HBM bound); the chain (N = 2^28),
  // FUSED with four steps per launch ahead of PLAIN (232 against 209 G site-steps/s); the
  // square lattice, PLAIN.  qw_plan_autotune re-measures on the device.
  if (stencil_supported(p->g, p->dtype, QW_STENCIL_TMA2)) return QW_STENCIL_TMA2;
  if (p->g.dim == 1 && fused_step_supported(p->g, p->dtype, p->fuse_depth, p->fuse_box)) return QW_STENCIL_FUSED;
  if (stencil_supported(p->g, p->dtype, QW_STENCIL_TMA)) return QW_STENCIL_TMA;
  if (stencil_supported(p->g, p->dtype, QW_STENCIL_VEC)) return QW_STENCIL_VEC;
  return QW_STENCIL_PLAIN;
}

static qw_status check_flags(qw_plan_s* p, cudaStream_t s) {
  // the error word lands in the last slot of the pinned result buffer (an asynchronous copy;
  // a pageable destination would be staged)
  int* flags = reinterpret_cast<int*>(p->red_host + 15);
  QW_CHECK_CUDA(cudaMemcpyAsync(flags, p->dev_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  QW_CHECK_CUDA(cudaStreamSynchronize(s));
  if (flags[0] != 0) {
    cudaMemsetAsync(p->dev_flags, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
    set_error("a bounded device wait gave up (code %d); results of the affected launch are invalid", flags[0]);
    return QW_ETIMEOUT;
  }
  return QW_OK;
}

static qw_status prepare_spectral(qw_plan_s* p) {
  if (p->spec_ready) return QW_OK;
  qw_status st = fft_plan_create(&p->fft, p->g, p->dtype);
  if (st != QW_OK) {
    fft_plan_destroy(&p->fft);
    return st;
  }
  // 8 bytes per stored wave vector (complex64: the split nu pair), 16 for complex128
  // (omega as a double-double); BCC stores q0 of each cell only
  QW_CHECK_CUDA(cudaMalloc(&p->omega, (p->dtype == QW_C64 ? 8 : 16) * p->g.vol));
  QW_CHECK_CUDA(cudaMalloc(&p->spec_partials, sizeof(double) * 2 * kObsBlocks));
  if (fused_x_supported(p->g, p->fft, p->dtype)) {
    QW_CHECK_CUDA(cudaMalloc(&p->xw_partials, sizeof(double) * 2 * (fused_x_grid(p->g) + kFoldCtas)));
    // the observables' first pass (outermost axis, from the field) also takes norm and <x>
    const int64_t ctas = fft_moment_ctas(p->fft, p->g.dim - 1);
    if (ctas > 0) {
      QW_CHECK_CUDA(cudaMalloc(&p->zm_partials, sizeof(double) * 4 * (ctas + kFoldCtas)));
      p->zm_ctas = ctas;
    }
  }
  st = launch_omega_table(p->g, spec_axes(p->g, p->fft), p->n, p->mass, p->omega, 0, p->dtype == QW_C64);
  if (st != QW_OK) return st;
  QW_CHECK_CUDA(cudaDeviceSynchronize());
  p->spec_ready = true;
  return QW_OK;
}

static qw_status use_device(const qw_plan_s* p) {
  int cur = -1;
  QW_CHECK_CUDA(cudaGetDevice(&cur));
  if (cur != p->device) QW_CHECK_CUDA(cudaSetDevice(p->device));
  return QW_OK;
}

}  // namespace qw

using namespace qw;

extern "C" {

const char* qw_last_error(void) { return g_last_error.c_str(); }

const char* qw_version(void) { return "qw-gb300 0.1 (sm_103a)"; }

qw_status qw_plan_create(int dim, int64_t N, double mass, qw_dtype dtype, qw_plan* out) {
  if (!out) {
    set_error("qw_plan_create: out is NULL");
    return QW_EINVAL;
  }
  *out = nullptr;
  Geometry g;
  if (!make_geometry(dim, N, &g)) {
    set_error("qw_plan_create: bad dim=%d / N=%lld (dim in 1..3, N >= 2, N even for dim 3)", dim, (long long)N);
    return QW_EINVAL;
  }
  if (!(mass >= 0.0 && mass <= 1.0)) {
    set_error("qw_plan_create: mass %g outside [0, 1]", mass);
    return QW_EINVAL;
  }
  if (dtype != QW_C64 && dtype != QW_C128) {
    set_error("qw_plan_create: bad dtype %d", (int)dtype);
    return QW_EINVAL;
  }
  qw_plan_s* p = new (std::nothrow) qw_plan_s();
  if (!p) {
    set_error("qw_plan_create: host allocation failed");
    return QW_ENOMEM;
  }
  p->g = g;
  p->mass = mass;
  p->n = std::sqrt(1.0 - mass * mass);
  p->dtype = dtype;
  p->elem_bytes = (dtype == QW_C64) ? 8 : 16;
  qw_status st = QW_OK;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaMalloc(&p->scratch, (size_t)g.elems * p->elem_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&p->red_partials, sizeof(double) * 10 * kMom2MaxBlocks);
  if (e == cudaSuccess) e = cudaMalloc(&p->red_result, sizeof(double) * 16);
  if (e == cudaSuccess) e = cudaMallocHost(&p->red_host, sizeof(double) * 16);
  if (e == cudaSuccess) e = cudaMalloc(&p->dev_flags, sizeof(int) * 2);
  if (e == cudaSuccess) e = cudaMemset(p->dev_flags, 0, sizeof(int) * 2);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    st = cuda_fail(e, "qw_plan_create: allocation");
    qw_plan_destroy(p);
    return st;
  }
  if (tma_step_supported(g) && dtype == QW_C64) {
    int nsm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
    std::vector<int4> items = tma_item_table(g, 2 * nsm, 4);
    if (e == cudaSuccess) e = cudaMalloc(&p->tma_items, items.size() * sizeof(int4));
    if (e == cudaSuccess)
      e = cudaMemcpy(p->tma_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
    p->tma_nitems = (int)items.size();
    if (e == cudaSuccess && tma2_step_supported(g)) {
      std::vector<int4> items2 = tma_item_table(g, nsm, 8);
      e = cudaMalloc(&p->tma2_items, items2.size() * sizeof(int4));
      if (e == cudaSuccess)
        e = cudaMemcpy(p->tma2_items, items2.data(), items2.size() * sizeof(int4), cudaMemcpyHostToDevice);
      p->tma2_nitems = (int)items2.size();
    }
    if (e != cudaSuccess) {
      st = cuda_fail(e, "qw_plan_create: TMA item tables");
      qw_plan_destroy(p);
      return st;
    }
  }
  // FUSED variant defaults: depth and tile box per lattice (qw_plan_autotune measures others)
  p->fuse_depth = g.dim == 3 ? 2 : 4;
  p->fuse_box[0] = g.dim == 1 ? 2048 : (g.dim == 2 ? 64 : 8);
  p->fuse_box[1] = g.dim == 1 ? 1 : (g.dim == 2 ? 16 : 8);
  p->fuse_box[2] = g.dim == 3 ? 6 : 1;
  p->stencil = default_stencil(p);
  *out = p;
  return QW_OK;
}

qw_status qw_plan_destroy(qw_plan p) {
  if (!p) return QW_OK;
  cudaDeviceSynchronize();
  if (p->scratch) cudaFree(p->scratch);
  if (p->red_partials) cudaFree(p->red_partials);
  if (p->red_result) cudaFree(p->red_result);
  if (p->red_host) cudaFreeHost(p->red_host);
  if (p->dev_flags) cudaFree(p->dev_flags);
  if (p->tma_items) cudaFree(p->tma_items);
  if (p->tma2_items) cudaFree(p->tma2_items);
  fft_plan_destroy(&p->fft);
  if (p->omega) cudaFree(p->omega);
  if (p->spec_partials) cudaFree(p->spec_partials);
  if (p->xw_partials) cudaFree(p->xw_partials);
  if (p->zm_partials) cudaFree(p->zm_partials);
  for (int b = 0; b < kHostBufs; ++b) {
    if (p->hbuf[b]) cudaFree(p->hbuf[b]);
    if (p->ev_copied[b]) cudaEventDestroy(p->ev_copied[b]);
    if (p->ev_freed[b]) cudaEventDestroy(p->ev_freed[b]);
    if (p->ev_stepped[b]) cudaEventDestroy(p->ev_stepped[b]);
  }
  if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
  for (cudaEvent_t e : p->tev) cudaEventDestroy(e);
  if (p->proj_partials) cudaFree(p->proj_partials);
  if (p->hstage) cudaFreeHost(p->hstage);
  delete p;
  return QW_OK;
}

int64_t qw_plan_field_elems(qw_plan p) { return p ? p->g.elems : -1; }

int64_t qw_plan_sites(qw_plan p) { return p ? p->g.sites : -1; }

qw_status qw_step(qw_plan p, void* psi, int64_t nsteps, void* stream) {
  NvtxRange nvtx_range("qw_step");
  if (!p || !psi || nsteps < 0) {
    set_error("qw_step: null plan/field or nsteps < 0");
    return QW_EINVAL;
  }
  if (nsteps == 0) return QW_OK;
  qw_status st = use_device(p);
  if (st != QW_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the VEC, TMA and TMA2 kernels move 16-byte vectors: a complex64 field that is only
  // 8-byte aligned (e.g. a view one element into an allocation) takes the PLAIN kernel
  const int variant = (aligned16(psi) || p->stencil == QW_STENCIL_FUSED) ? p->stencil : QW_STENCIL_PLAIN;
  if (debug_poison())
    QW_CHECK_CUDA(cudaMemsetAsync(p->scratch, kPoisonByte, (size_t)p->g.elems * p->elem_bytes, s));
  void* cur = psi;
  void* nxt = p->scratch;
  for (int64_t i = 0; i < nsteps;) {
    int done = 1;
    if (variant == QW_STENCIL_TMA2 && nsteps - i >= 2) {
      st = launch_step_tma2(p->g, p->n, p->mass, cur, nxt, p->tma2_items, p->tma2_nitems, p->dev_flags,
                            p->dev_flags + 1, s);
      done = 2;
    } else if (variant == QW_STENCIL_TMA || variant == QW_STENCIL_TMA2) {
      st = launch_step_tma(p->g, p->n, p->mass, cur, nxt, p->tma_items, p->tma_nitems, p->dev_flags,
                           p->dev_flags + 1, s);
    } else if (variant == QW_STENCIL_FUSED) {
      done = (int)std::min<int64_t>(p->fuse_depth, nsteps - i);
      st = launch_step_fused(p->g, p->fuse_depth, p->fuse_box, done, p->n, p->mass, cur, nxt, s);
    } else {
      st = launch_step(p->g, p->dtype, variant, p->n, p->mass, cur, nxt, s);
    }
    if (st != QW_OK) return st;
    void* t = cur;
    cur = nxt;
    nxt = t;
    i += done;
  }
  if (cur != psi)
    QW_CHECK_CUDA(cudaMemcpyAsync(psi, cur, (size_t)p->g.elems * p->elem_bytes, cudaMemcpyDeviceToDevice, s));
  return QW_OK;
}

qw_status qw_plan_set_stencil(qw_plan p, int variant) {
  if (!p) {
    set_error("qw_plan_set_stencil: null plan");
    return QW_EINVAL;
  }
  if (variant == QW_STENCIL_AUTO) {
    p->stencil = default_stencil(p);
    return QW_OK;
  }
  if (variant == QW_STENCIL_FUSED ? !fused_step_supported(p->g, p->dtype, p->fuse_depth, p->fuse_box)
                                  : !stencil_supported(p->g, p->dtype, variant)) {
    set_error("qw_plan_set_stencil: variant %d does not support dim=%d N=%lld dtype=%d", variant, p->g.dim,
              (long long)p->g.N, (int)p->dtype);
    return QW_EINVAL;
  }
  p->stencil = variant;
  return QW_OK;
}

int qw_plan_get_stencil(qw_plan p) { return p ? p->stencil : -1; }

qw_status qw_plan_prepare_spectral(qw_plan p) {
  NvtxRange nvtx_range("qw_plan_prepare_spectral");
  if (!p) {
    set_error("qw_plan_prepare_spectral: null plan");
    return QW_EINVAL;
  }
  qw_status st = use_device(p);
  if (st != QW_OK) return st;
  return prepare_spectral(p);
}

qw_status qw_evolve_spectral(qw_plan p, void* psi, int64_t t, void* stream) {
  NvtxRange nvtx_range("qw_evolve_spectral");
  if (!p || !psi || t < 0) {
    set_error("qw_evolve_spectral: null plan/field or t < 0");
    return QW_EINVAL;
  }
  qw_status st = use_device(p);
  if (st != QW_OK) return st;
  st = prepare_spectral(p);
  if (st != QW_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (fused_x_supported(p->g, p->fft, p->dtype)) {
    // y, z forward; x forward + D_k^t + x inverse in one pass; y, z inverse
    for (int ax = p->g.dim - 1; ax >= 1; --ax)
      if ((st = fft_forward_axis(p->fft, ax, psi, s)) != QW_OK) return st;
    st = launch_evolve_fused_x(p->g, spec_axes(p->g, p->fft), p->fft, p->n, p->mass, p->omega, t, psi, s);
    if (st != QW_OK) return st;
    for (int ax = 1; ax < p->g.dim; ++ax)
      if ((st = fft_inverse_axis(p->fft, ax, psi, s)) != QW_OK) return st;
    return QW_OK;
  }
  st = fft_forward(p->fft, p->g.dim, psi, s);
  if (st != QW_OK) return st;
  st = launch_evolve_pointwise(p->g, spec_axes(p->g, p->fft), p->dtype, p->n, p->mass, p->omega, t, psi, s);
  if (st != QW_OK) return st;
  return fft_inverse(p->fft, p->g.dim, psi, s);
}

qw_status qw_prepare_packet(qw_plan p, void* psi, const double* x0, double sigma, const double* k0,
                            const double* chi, void* stream) {
  NvtxRange nvtx_range("qw_prepare_packet");
  if (!p || !psi || !x0 || !k0 || !chi) {
    set_error("qw_prepare_packet: null argument");
    return QW_EINVAL;
  }
  qw_status st = use_device(p);
  if (st != QW_OK) return st;
  return launch_packet(p->g, p->dtype, x0, sigma, k0, chi, psi, static_cast<cudaStream_t>(stream));
}

qw_status qw_plan_autotune(qw_plan p, void* stream, double* best_rate) {
  NvtxRange nvtx_range("qw_plan_autotune");
  if (!p) {
    set_error("qw_plan_autotune: null plan");
    return QW_EINVAL;
  }
  qw_status st = use_device(p);
  if (st != QW_OK) return st;
  char problem[96];
  std::snprintf(problem, sizeof(problem), "dim=%d N=%lld dtype=%s", p->g.dim, (long long)p->g.N,
                p->dtype == QW_C64 ? "c64" : "c128");
  std::vector<double> cached;
  if (autotune_cache_get("plan", problem, &cached) && cached.size() == 6) {
    const int v = (int)cached[0], dpt = (int)cached[1];
    const int box[3] = {(int)cached[2], (int)cached[3], (int)cached[4]};
    const bool ok = v == QW_STENCIL_FUSED ? fused_step_supported(p->g, p->dtype, dpt, box)
                                          : (v >= QW_STENCIL_PLAIN && v <= QW_STENCIL_TMA2 &&
                                             stencil_supported(p->g, p->dtype, v));
    if (ok) {  // the measured choice of an earlier run on this GPU model
      p->stencil = v;
      if (v == QW_STENCIL_FUSED) {
        p->fuse_depth = dpt;
        for (int a = 0; a < 3; ++a) p->fuse_box[a] = box[a];
      }
      if (best_rate) *best_rate = cached[5];
      return QW_OK;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* tmp = nullptr;
  const size_t bytes = (size_t)p->g.elems * p->elem_bytes;
  QW_CHECK_CUDA(cudaMalloc(&tmp, bytes));
  QW_CHECK_CUDA(cudaMemsetAsync(tmp, 0, bytes, s));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int saved = p->stencil, saved_depth = p->fuse_depth;
  const int saved_box[3] = {p->fuse_box[0], p->fuse_box[1], p->fuse_box[2]};
  int best = saved, best_depth = saved_depth, best_box[3] = {saved_box[0], saved_box[1], saved_box[2]};
  double best_r = -1.0;
  // candidates: the data-movement variants, then FUSED with depth 2..4 and a few tile boxes
  struct Cand {
    int v, depth, box[3];
  };
  std::vector<Cand> cands;
  for (int v : {QW_STENCIL_PLAIN, QW_STENCIL_VEC, QW_STENCIL_TMA, QW_STENCIL_TMA2}) cands.push_back({v, 0, {0, 0, 0}});
  const int boxes[3][3][3] = {{{1024, 1, 1}, {2048, 1, 1}, {4096, 1, 1}},
                              {{32, 16, 1}, {64, 16, 1}, {64, 8, 1}},
                              {{8, 8, 4}, {8, 8, 6}, {16, 8, 4}}};
  for (int dpt = 2; dpt <= 4; ++dpt)
    for (int k = 0; k < 3; ++k) {
      const int* b = boxes[p->g.dim - 1][k];
      cands.push_back({QW_STENCIL_FUSED, dpt, {b[0], b[1], b[2]}});
    }
  const int64_t steps = 8;
  for (const Cand& c : cands) {
    if (c.v == QW_STENCIL_FUSED ? !fused_step_supported(p->g, p->dtype, c.depth, c.box)
                                : !stencil_supported(p->g, p->dtype, c.v))
      continue;
    p->stencil = c.v;
    if (c.v == QW_STENCIL_FUSED) {
      p->fuse_depth = c.depth;
      for (int a = 0; a < 3; ++a) p->fuse_box[a] = c.box[a];
    }
    st = qw_step(p, tmp, 2, s);  // warm-up
    if (st != QW_OK) break;
    cudaEventRecord(e0, s);
    st = qw_step(p, tmp, steps, s);
    cudaEventRecord(e1, s);
    if (st != QW_OK) break;
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double r = (double)p->g.sites * steps / (ms * 1e-3);
    if (r > best_r) {
      best_r = r;
      best = c.v;
      if (c.v == QW_STENCIL_FUSED) {
        best_depth = c.depth;
        for (int a = 0; a < 3; ++a) best_box[a] = c.box[a];
      }
    }
  }
  p->fuse_depth = st == QW_OK ? best_depth : saved_depth;
  for (int a = 0; a < 3; ++a) p->fuse_box[a] = st == QW_OK ? best_box[a] : saved_box[a];
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(tmp);
  p->stencil = (st == QW_OK) ? best : saved;
  if (best_rate) *best_rate = best_r;
  if (st != QW_OK) return st;
  st = check_flags(p, s);
  if (st == QW_OK)
    autotune_cache_put("plan", problem, {(double)best, (double)best_depth, (double)best_box[0], (double)best_box[1],
                                         (double)best_box[2], best_r});
  return st;
}

qw_status qw_sync(qw_plan p, void* stream) {
  if (!p) {
    set_error("qw_sync: null plan");
    return QW_EINVAL;
  }
  qw_status st = use_device(p);
  if (st != QW_OK) return st;
  return check_flags(p, static_cast<cudaStream_t>(stream));
}

// Observables of psi: the reductions are enqueued on s, then obs_finish waits for them
// and fills *out.  kspace: whether the particle weights are computed (axis lengths 2^a 3^b).
static qw_status obs_enqueue(qw_plan_s* p, const void* psi, cudaStream_t s, double* host_dst, bool* kspace_out) {
  if (debug_poison())
    QW_CHECK_CUDA(cudaMemsetAsync(p->scratch, kPoisonByte, (size_t)p->g.elems * p->elem_bytes, s));
  // particle weights need the spectrum (computed into the scratch field)
  const bool kspace = fft_size_ok(p->g.nx) && fft_size_ok(p->g.ny) && fft_size_ok(p->g.nz);
  *kspace_out = kspace;
  qw_status st = QW_OK;
  if (kspace) {
    st = prepare_spectral(p);
    if (st != QW_OK) return st;
  }
  if (!(kspace && p->xw_partials && p->zm_ctas > 0)) {
    st = launch_position_moments(p->g, p->dtype, psi, p->red_partials, p->red_result, s);
    if (st != QW_OK) return st;
  }
  if (kspace) {
    const SpecAxes ax = spec_axes(p->g, p->fft);
    if (p->xw_partials) {
      // the outermost axis reads psi and writes the scratch field (taking norm and <x> of psi
      // on the way where it can), the middle axis works in place, and the x transform is done
      // in shared memory by the weights kernel itself
      if (p->zm_ctas > 0) {
        const FftMoments mom{p->g.dim, (int)p->g.nx, p->g.s, p->zm_partials};
        st = fft_forward_axis_from_moments(p->fft, p->g.dim - 1, psi, p->scratch, mom, s);
        if (st == QW_OK)
          st = launch_fold_partials(p->zm_partials, p->zm_ctas, 4, p->zm_partials + 4 * p->zm_ctas, p->red_result, s);
      } else {
        st = fft_forward_axis_from(p->fft, p->g.dim - 1, psi, p->scratch, s);
      }
      for (int a = p->g.dim - 2; a >= 1 && st == QW_OK; --a) st = fft_forward_axis(p->fft, a, p->scratch, s);
      if (st != QW_OK) return st;
      st = launch_weights_fused_x(p->g, ax, p->fft, p->n, p->mass, p->scratch, p->xw_partials, p->red_result + 4, s);
      if (st != QW_OK) return st;
    } else {
      // particle weights need the spectrum: forward DFT of a copy in the scratch field
      QW_CHECK_CUDA(
          cudaMemcpyAsync(p->scratch, psi, (size_t)p->g.elems * p->elem_bytes, cudaMemcpyDeviceToDevice, s));
      st = fft_forward(p->fft, p->g.dim, p->scratch, s);
      if (st != QW_OK) return st;
      st = launch_particle_weights(p->g, ax, p->dtype, p->n, p->mass, p->scratch, p->spec_partials,
                                   p->red_result + 4, s);
      if (st != QW_OK) return st;
    }
  }
  QW_CHECK_CUDA(cudaMemcpyAsync(host_dst, p->red_result, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
  return QW_OK;
}

// *out from the six reduced sums r (norm, three first moments, the two weight sums).
static void obs_fill(const qw_plan_s* p, const double* r, bool kspace, qw_obs* out) {
  out->norm = r[0];
  for (int j = 0; j < 3; ++j) out->x_mean[j] = (j < p->g.dim && r[0] > 0) ? r[1 + j] / r[0] : 0.0;
  if (kspace && r[4] > 0) {
    out->w_particle = 0.5 * (1.0 + r[5] / r[4]);
    out->w_antiparticle = 0.5 * (1.0 - r[5] / r[4]);
  } else {
    out->w_particle = NAN;
    out->w_antiparticle = NAN;
  }
}

qw_status qw_observables(qw_plan p, const void* psi, qw_obs* out, void* stream) {
  NvtxRange nvtx_range("qw_observables");
  if (!p || !psi || !out) {
    set_error("qw_observables: null argument");
    return QW_EINVAL;
  }
  qw_status st = use_device(p);
  if (st != QW_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bool kspace = false;
  st = obs_enqueue(p, psi, s, p->red_host, &kspace);
  if (st != QW_OK) return st;
  st = check_flags(p, s);  // waits for the stream
  if (st != QW_OK) return st;
  obs_fill(p, p->red_host, kspace, out);
  return QW_OK;
}

qw_status qw_fw_transform(qw_plan p, const void* psi, void* out, void* stream) {
  NvtxRange nvtx_range("qw_fw_transform");
  if (!p || !psi || !out) {
    set_error("qw_fw_transform: null argument");
    return QW_EINVAL;
  }
  qw_status st = use_device(p);
  if (st != QW_OK) return st;
  st = prepare_spectral(p);
  if (st != QW_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (out != psi)
    QW_CHECK_CUDA(cudaMemcpyAsync(out, psi, (size_t)p->g.elems * p->elem_bytes, cudaMemcpyDeviceToDevice, s));
  if ((st = fft_forward(p->fft, p->g.dim, out, s)) != QW_OK) return st;
  if ((st = launch_fw_pointwise(p->g, spec_axes(p->g, p->fft), p->dtype, p->n, p->mass, out, s)) != QW_OK) return st;
  return fft_inverse(p->fft, p->g.dim, out, s);
}

qw_status qw_position_moments(qw_plan p, const void* psi, double* out, void* stream) {
  NvtxRange nvtx_range("qw_position_moments");
  if (!p || !psi || !out) {
    set_error("qw_position_moments: null argument");
    return QW_EINVAL;
  }
  qw_status st = use_device(p);
  if (st != QW_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = launch_position_moments2(p->g, p->dtype, psi, p->red_partials, p->red_result, s);
  if (st != QW_OK) return st;
  QW_CHECK_CUDA(cudaMemcpyAsync(p->red_host, p->red_result, 10 * sizeof(double), cudaMemcpyDeviceToHost, s));
  st = check_flags(p, s);  // waits for the stream
  if (st != QW_OK) return st;
  const double* r = p->red_host;
  const double n = r[0];
  out[0] = n;
  double mu[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < 3; ++i) mu[i] = (i < p->g.dim && n > 0) ? r[1 + i] / n : 0.0;
  for (int i = 0; i < 3; ++i) out[1 + i] = mu[i];
  // central moments E[X_i X_j] - mu_i mu_j, axes at or above dim are 0
  const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
  for (int q = 0; q < 6; ++q)
    out[4 + q] = (ii[q] < p->g.dim && jj[q] < p->g.dim && n > 0) ? r[4 + q] / n - mu[ii[q]] * mu[jj[q]] : 0.0;
  return QW_OK;
}

qw_status qw_projection(qw_plan p, const void* psi, int keep, double* out, void* stream) {
  NvtxRange nvtx_range("qw_projection");
  if (!p || !psi || !out) {
    set_error("qw_projection: null argument");
    return QW_EINVAL;
  }
  if (keep <= 0 || keep >= (1 << p->g.dim)) {
    set_error("qw_projection: keep mask %d must name 1..%d of the axes below dim %d", keep, p->g.dim, p->g.dim);
    return QW_EINVAL;
  }
  qw_status st = use_device(p);
  if (st != QW_OK) return st;
  const int64_t need = projection_partials(p->g, keep, p->dtype);
  if (need > p->proj_cap) {
    if (p->proj_partials) QW_CHECK_CUDA(cudaFree(p->proj_partials));
    p->proj_partials = nullptr;
    p->proj_cap = 0;
    QW_CHECK_CUDA(cudaMalloc(&p->proj_partials, sizeof(double) * need));
    p->proj_cap = need;
  }
  return launch_projection(p->g, p->dtype, psi, keep, out, p->proj_partials, static_cast<cudaStream_t>(stream));
}

int64_t qw_projection_elems(qw_plan p, int keep) {
  if (!p || keep <= 0 || keep >= (1 << p->g.dim)) return -1;
  return projection_outputs(p->g, keep);
}

// Two device fields, a non-blocking copy stream and its events for qw_run_host.
static qw_status host_run_setup(qw_plan_s* p) {
  if (p->copy_stream) return QW_OK;
  const size_t bytes = (size_t)p->g.elems * p->elem_bytes;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < kHostBufs && e == cudaSuccess; ++b) {
    // written once here, so that a run's first copy into each buffer is not the first
    // write into freshly allocated device memory
    if (!p->hbuf[b]) {
      e = cudaMalloc(&p->hbuf[b], bytes);
      if (e == cudaSuccess) e = cudaMemset(p->hbuf[b], 0, bytes);
    }
    if (e == cudaSuccess && !p->ev_copied[b]) e = cudaEventCreateWithFlags(&p->ev_copied[b], cudaEventDisableTiming);
    if (e == cudaSuccess && !p->ev_freed[b]) e = cudaEventCreateWithFlags(&p->ev_freed[b], cudaEventDisableTiming);
    if (e == cudaSuccess && !p->ev_stepped[b])
      e = cudaEventCreateWithFlags(&p->ev_stepped[b], cudaEventDisableTiming);
  }
  if (e == cudaSuccess && !p->hstage) e = cudaMallocHost(&p->hstage, sizeof(double) * 16);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaGetLastError();
    const qw_status st = (e == cudaErrorMemoryAllocation) ? QW_ENOMEM : QW_ECUDA;
    set_error("qw_run_host: device buffers / copy stream: %s", cudaGetErrorString(e));
    p->copy_stream = nullptr;
    return st;
  }
  return QW_OK;
}

qw_status qw_run_host(qw_plan p, const void* const* psi_host, void* const* psi_out_host, int count, int64_t nsteps,
                      qw_obs* out, void* stream) {
  NvtxRange nvtx_range("qw_run_host");
  if (!p || count < 0 || nsteps < 0 || (count > 0 && (!psi_host || !out))) {
    set_error("qw_run_host: null plan/array, count < 0 or nsteps < 0");
    return QW_EINVAL;
  }
  for (int j = 0; j < count; ++j)
    if (!psi_host[j] || (psi_out_host && !psi_out_host[j])) {
      set_error("qw_run_host: null field pointer at index %d", j);
      return QW_EINVAL;
    }
  if (count == 0) return QW_OK;
  qw_status st = use_device(p);
  if (st != QW_OK) return st;
  st = host_run_setup(p);
  if (st != QW_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream), cs = p->copy_stream;
  const size_t bytes = (size_t)p->g.elems * p->elem_bytes;
  // field j lives in hbuf[j % NB] (NB = kHostBufs = 3); on the copy stream: in(0), in(1),
  // then per field j: in(j + 2), out(j).  in(j + 2) waits for field j - 1's observables (its
  // buffer's previous field) and follows out(j - 1) in stream order, so it overlaps field j's
  // step and has until field j + 2's step to land.  Field j's sums go to the pinned stage
  // j % 2; the host reads them only after field j + 1's step is enqueued, so the device never
  // waits for the host between fields.
  constexpr int NB = kHostBufs;
  const bool timing = p->host_timing;
  if (timing) {
    while ((int)p->tev.size() < 5 * count) {
      cudaEvent_t e;
      QW_CHECK_CUDA(cudaEventCreate(&e));
      p->tev.push_back(e);
    }
    p->tev_fields = 0;
  }
  // timing event i of field j (no-op unless timing is on)
  auto mark = [&](int j, int i, cudaStream_t on) -> cudaError_t {
    return timing ? cudaEventRecord(p->tev[5 * j + i], on) : cudaSuccess;
  };
  // the copy of field k into its buffer, with its completion event
  auto copy_in = [&](int k) -> qw_status {
    const int kb = k % NB;
    QW_CHECK_CUDA(mark(k, 0, cs));
    QW_CHECK_CUDA(cudaMemcpyAsync(p->hbuf[kb], psi_host[k], bytes, cudaMemcpyHostToDevice, cs));
    QW_CHECK_CUDA(mark(k, 1, cs));
    QW_CHECK_CUDA(cudaEventRecord(p->ev_copied[kb], cs));
    return QW_OK;
  };
  for (int k = 0; k < NB - 1 && k < count; ++k)
    if ((st = copy_in(k)) != QW_OK) return st;
  bool kspace = false;
  int done = 0;  // fields whose observables are on the host
  for (int j = 0; j < count && st == QW_OK; ++j) {
    const int b = j % NB;
    if (j + NB - 1 < count) {
      // field j + NB - 1 reuses field j - 1's buffer (none before the first field)
      if (j >= 1) QW_CHECK_CUDA(cudaStreamWaitEvent(cs, p->ev_freed[(j - 1) % NB], 0));
      if ((st = copy_in(j + NB - 1)) != QW_OK) break;
    }
    QW_CHECK_CUDA(cudaStreamWaitEvent(s, p->ev_copied[b], 0));
    QW_CHECK_CUDA(mark(j, 2, s));
    st = qw_step(p, p->hbuf[b], nsteps, stream);
    if (st != QW_OK) break;
    QW_CHECK_CUDA(mark(j, 3, s));
    if (psi_out_host) {
      QW_CHECK_CUDA(cudaEventRecord(p->ev_stepped[b], s));
      QW_CHECK_CUDA(cudaStreamWaitEvent(cs, p->ev_stepped[b], 0));
      QW_CHECK_CUDA(cudaMemcpyAsync(psi_out_host[j], p->hbuf[b], bytes, cudaMemcpyDeviceToHost, cs));
    }
    st = obs_enqueue(p, p->hbuf[b], s, p->hstage + 8 * (j & 1), &kspace);
    if (st != QW_OK) break;
    QW_CHECK_CUDA(cudaEventRecord(p->ev_freed[b], s));
    QW_CHECK_CUDA(mark(j, 4, s));
    if (timing) p->tev_fields = j + 1;
    if (j >= 1) {  // the previous field's sums
      const cudaError_t e = cudaEventSynchronize(p->ev_freed[(j - 1) % NB]);
      if (e != cudaSuccess) {
        st = cuda_fail(e, "qw_run_host: observables");
        break;
      }
      obs_fill(p, p->hstage + 8 * ((j - 1) & 1), kspace, &out[j - 1]);
      done = j;
    }
  }
  // the last field's sums, the device error word, and every copy (the last read-back
  // included) before the host buffers are handed back
  const qw_status sf = check_flags(p, s);
  if (st == QW_OK) st = sf;
  if (st == QW_OK && done == count - 1) obs_fill(p, p->hstage + 8 * ((count - 1) & 1), kspace, &out[count - 1]);
  const cudaError_t e = cudaStreamSynchronize(cs);
  if (st == QW_OK && e != cudaSuccess) return cuda_fail(e, "qw_run_host: copy stream");
  return st;
}

qw_status qw_plan_set_host_timing(qw_plan p, int on) {
  if (!p) {
    set_error("qw_plan_set_host_timing: null plan");
    return QW_EINVAL;
  }
  p->host_timing = on != 0;
  return QW_OK;
}

qw_status qw_plan_host_timing(qw_plan p, double* out, int count) {
  if (!p || !out || count < 1 || count > p->tev_fields) {
    set_error("qw_plan_host_timing: null argument, or count outside 1..%d (fields of the last timed run)",
              p ? p->tev_fields : 0);
    return QW_EINVAL;
  }
  qw_status st = use_device(p);
  if (st != QW_OK) return st;
  QW_CHECK_CUDA(cudaEventSynchronize(p->tev[5 * (count - 1) + 4]));
  for (int j = 0; j < count; ++j)
    for (int i = 0; i < 5; ++i) {
      float ms = 0.f;
      QW_CHECK_CUDA(cudaEventElapsedTime(&ms, p->tev[0], p->tev[5 * j + i]));
      out[5 * j + i] = ms;
    }
  return QW_OK;
}

qw_status qw_plan_set_fusion(qw_plan p, int depth, const int* box) {
  if (!p || !box || !fused_step_supported(p->g, p->dtype, depth, box)) {
    set_error("qw_plan_set_fusion: null argument, or depth %d / this box not supported for the plan "
              "(complex64, depth 2..4, the tile and its halo in 227 KB of shared memory)",
              depth);
    return QW_EINVAL;
  }
  p->fuse_depth = depth;
  for (int a = 0; a < 3; ++a) p->fuse_box[a] = a < p->g.dim ? box[a] : 1;
  return QW_OK;
}

qw_status qw_plan_get_fusion(qw_plan p, int* depth, int* box) {
  if (!p) {
    set_error("qw_plan_get_fusion: null plan");
    return QW_EINVAL;
  }
  if (depth) *depth = p->fuse_depth;
  if (box)
    for (int a = 0; a < 3; ++a) box[a] = p->fuse_box[a];
  return QW_OK;
}

qw_status qw_set_autotune_cache(const char* path) {
  std::lock_guard<std::mutex> lock(g_cache_mu);
  g_cache_path = path ? path : "";
  return QW_OK;
}

qw_status qw_set_debug_poison(int on) {
  g_poison.store(on != 0, std::memory_order_relaxed);
  return QW_OK;
}

}  // extern "C"
