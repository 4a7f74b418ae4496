// Serving: walk requests evolved in the Fourier form of Sec. 4 with continuous
// batching.
//
// qw_submit copies a request into a pending FIFO and returns a ticket.  One
// scheduler thread owns all device work:
//   * admission: the head of the FIFO is admitted as soon as an execution slot
//     (a CUDA stream) is free and its fields fit in the device pool, whose size
//     is the server's HBM budget (allocated once: the loop never calls cudaMalloc);
//     the FFT tables of each box size are carved from the same pool (generated on
//     the device, counted in bytes_in_use), cached while the pool has room, and
//     evicted least recently used first when an admission needs the space;
//   * an admitted request runs on its slot's stream: initial state (Gaussian
//     packet built on the device, or the caller's field copied at submit), its
//     norm, forward FFT, D_k^t (normalised; omega_k in FP64 inside the kernel),
//     the particle weights on the evolved spectrum, inverse FFT, then <x> and
//     norm; ten doubles come back into pinned host memory and an event marks the end;
//   * completion: finished slots give their memory and stream back, so requests
//     that arrived meanwhile are admitted while others are still on the GPU.
// Requests in different slots overlap on the device.  qw_poll reads a ticket's
// state and, once done, the observables and the submit-to-done latency.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <new>
#include <thread>
#include <vector>

#include "qw_internal.cuh"

namespace qw {

using Clock = std::chrono::steady_clock;

// First-fit sub-allocator over one device block (offsets aligned to 256 bytes).
class Pool {
 public:
  void init(size_t bytes) {
    free_.clear();
    free_[0] = bytes;
    size_ = bytes;
    used_ = peak_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        if (used_ > peak_) peak_ = used_;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t size() const { return size_; }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0, used_ = 0, peak_ = 0;
};

enum TicketState { T_PENDING = 0, T_RUNNING = 1, T_DONE = 2, T_FAILED = 3 };

struct Request {
  uint64_t ticket;
  qw_request req;
  std::vector<unsigned char> psi0;  // copy of the caller's field, if any
  Clock::time_point t_submit;
  Geometry g;
  size_t bytes_field = 0, bytes_omega = 0;
  size_t bytes_tables = 0;  // FFT tables of this box size, if not cached at admission
};

// FFT plan of one box size whose tables live in the pool.
struct CachedFft {
  FftPlan plan;
  size_t off = 0, bytes = 0;
  int users = 0;              // admitted requests using it
  uint64_t last_use = 0;
  cudaEvent_t ready = nullptr;  // recorded after the table kernels on the creating stream
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  double* d_res = nullptr;       // 4 moments of psi(0), 4 moments of psi(t), 2 weights
  double* d_part = nullptr;      // partial sums
  double* h_res = nullptr;       // pinned copy of d_res
  bool busy = false;
  std::unique_ptr<Request> r;
  size_t off = 0, bytes = 0;
  CachedFft* fft = nullptr;
};

struct Result {
  TicketState state = T_PENDING;
  qw_obs obs;
  double latency = 0.0;
  std::string error;
};

}  // namespace qw

using namespace qw;

struct qw_server_s {
  int device = 0;
  size_t budget = 0;
  void* pool_base = nullptr;
  Pool pool;
  std::vector<Slot> slots;
  size_t max_pending = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::unique_ptr<Request>> pending;
  std::map<uint64_t, Result> results;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  std::map<std::pair<int, int64_t>, std::unique_ptr<CachedFft>> ffts;  // per box size (complex64)
  uint64_t use_clock = 0;
  uint64_t admitted = 0, completed = 0;
};

namespace qw {

static size_t request_bytes(const Geometry& g, size_t* field, size_t* omega) {
  *field = (size_t)g.elems * 8;  // complex64
  *omega = 0;                    // omega_k is computed inside the evolve kernel
  return ((*field + 255) & ~size_t(255)) + ((*omega + 255) & ~size_t(255));
}

// Drop the least recently used cached plan that no admitted request uses (not `keep`);
// false if there is none.  Called with the server lock held.
static bool evict_one_fft(qw_server_s* S, const CachedFft* keep) {
  auto victim = S->ffts.end();
  for (auto it = S->ffts.begin(); it != S->ffts.end(); ++it) {
    if (it->second->users > 0 || it->second.get() == keep) continue;
    if (victim == S->ffts.end() || it->second->last_use < victim->second->last_use) victim = it;
  }
  if (victim == S->ffts.end()) return false;
  S->pool.release(victim->second->off, victim->second->bytes);
  if (victim->second->ready) cudaEventDestroy(victim->second->ready);
  S->ffts.erase(victim);
  return true;
}

// Pool space for the head request: its field, plus its box size's FFT tables when they
// are not cached.  Evicts idle cached plans while the pool is short.  On success the
// slot holds the field's offset and the plan (created, tables generated on the slot's
// stream, when new); false leaves the request pending.  Called with the server lock held.
static bool admit_memory(qw_server_s* S, Request& R, Slot& sl, qw_status* st) {
  *st = QW_OK;
  const auto key = std::make_pair(R.g.dim, R.g.N);
  auto it = S->ffts.find(key);
  CachedFft* cf = it == S->ffts.end() ? nullptr : it->second.get();
  const size_t need = R.bytes_field + R.bytes_omega + 512;
  size_t off = 0, toff = 0;
  for (;;) {
    if (S->pool.alloc(need, &off)) {
      if (cf || S->pool.alloc(R.bytes_tables, &toff)) break;
      S->pool.release(off, need);
    }
    if (!evict_one_fft(S, cf)) return false;
  }
  if (!cf) {
    std::unique_ptr<CachedFft> c(new (std::nothrow) CachedFft());
    cudaError_t e = c ? cudaEventCreateWithFlags(&c->ready, cudaEventDisableTiming) : cudaErrorMemoryAllocation;
    if (e == cudaSuccess) {
      TableDst dst;
      dst.base = static_cast<char*>(S->pool_base) + toff;
      dst.cap = R.bytes_tables;
      dst.st = sl.stream;
      *st = fft_plan_create(&c->plan, R.g, QW_C64, &dst);
      if (*st == QW_OK) e = cudaEventRecord(c->ready, sl.stream);
    }
    if (e != cudaSuccess && *st == QW_OK) *st = cuda_fail(e, "served request: FFT tables");
    if (*st != QW_OK) {
      if (c && c->ready) cudaEventDestroy(c->ready);
      S->pool.release(toff, R.bytes_tables);
      S->pool.release(off, need);
      return true;  // admitted as failed: the caller finishes it with *st
    }
    c->off = toff;
    c->bytes = R.bytes_tables;
    cf = c.get();
    S->ffts[key] = std::move(c);
  }
  cf->users++;
  cf->last_use = ++S->use_clock;
  sl.fft = cf;
  sl.off = off;
  sl.bytes = need;
  return true;
}

// Enqueue the whole request on the slot's stream.
static qw_status launch_request(qw_server_s* S, Slot& sl) {
  NvtxRange nvtx_range("qw_server request launch");
  Request& R = *sl.r;
  const Geometry& g = R.g;
  cudaStream_t s = sl.stream;
  char* base = static_cast<char*>(S->pool_base) + sl.off;
  void* psi = base;
  const double m = R.req.mass, n = std::sqrt(1.0 - m * m);
  qw_status st;
  const FftPlan* f = &sl.fft->plan;
  // tables generated on another slot's stream must be complete first
  QW_CHECK_CUDA(cudaStreamWaitEvent(s, sl.fft->ready, 0));
  const SpecAxes ax = spec_axes(g, *f);
  if (!R.psi0.empty()) {
    QW_CHECK_CUDA(cudaMemcpyAsync(psi, R.psi0.data(), R.bytes_field, cudaMemcpyHostToDevice, s));
  } else {
    st = launch_packet(g, QW_C64, R.req.x0, R.req.sigma, R.req.k0, R.req.chi, psi, s);
    if (st != QW_OK) return st;
  }
  // norm of the initial state (its first moment slot), used to normalise
  if ((st = launch_position_moments(g, QW_C64, psi, sl.d_part, sl.d_res, s)) != QW_OK) return st;
  if ((st = fft_forward(*f, g.dim, psi, s)) != QW_OK) return st;
  // D_k^t with omega_k computed in the kernel (a request's table would be used once)
  if ((st = launch_evolve_pointwise(g, ax, QW_C64, n, m, nullptr, R.req.t, psi, s, sl.d_res)) != QW_OK) return st;
  // particle weights from the evolved spectrum: |P(+-) psi^_k|^2 is what a forward
  // DFT of psi(t) would give (the ratio does not depend on the DFT's scale)
  if ((st = launch_particle_weights(g, ax, QW_C64, n, m, psi, sl.d_part, sl.d_res + 8, s)) != QW_OK) return st;
  if ((st = fft_inverse(*f, g.dim, psi, s)) != QW_OK) return st;
  if ((st = launch_position_moments(g, QW_C64, psi, sl.d_part, sl.d_res + 4, s)) != QW_OK) return st;
  QW_CHECK_CUDA(cudaMemcpyAsync(sl.h_res, sl.d_res, 10 * sizeof(double), cudaMemcpyDeviceToHost, s));
  QW_CHECK_CUDA(cudaEventRecord(sl.done, s));
  return QW_OK;
}

static void finish_slot(qw_server_s* S, Slot& sl, qw_status st) {
  Request& R = *sl.r;
  Result res;
  res.latency = std::chrono::duration<double>(Clock::now() - R.t_submit).count();
  if (st == QW_OK) {
    const double* h = sl.h_res + 4;
    res.state = T_DONE;
    res.obs.norm = h[0];
    for (int j = 0; j < 3; ++j) res.obs.x_mean[j] = (j < R.g.dim && h[0] > 0) ? h[1 + j] / h[0] : 0.0;
    const double* w = sl.h_res + 8;
    res.obs.w_particle = w[0] > 0 ? 0.5 * (1.0 + w[1] / w[0]) : NAN;
    res.obs.w_antiparticle = w[0] > 0 ? 0.5 * (1.0 - w[1] / w[0]) : NAN;
  } else {
    res.state = T_FAILED;
    res.error = qw_last_error();
  }
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (sl.bytes) S->pool.release(sl.off, sl.bytes);
    if (sl.fft) sl.fft->users--;
    S->results[R.ticket] = res;
    S->completed++;
  }
  sl.fft = nullptr;
  sl.bytes = 0;
  sl.r.reset();
  sl.busy = false;
}

static void worker_loop(qw_server_s* S) {
  cudaSetDevice(S->device);
  for (;;) {
    bool idle = true;
    // completions
    for (auto& sl : S->slots) {
      if (!sl.busy) continue;
      cudaError_t e = cudaEventQuery(sl.done);
      if (e == cudaErrorNotReady) continue;
      idle = false;
      finish_slot(S, sl, e == cudaSuccess ? QW_OK : cuda_fail(e, "served request"));
    }
    // admissions (FIFO head first, as long as a slot and pool memory are free)
    for (;;) {
      Slot* free_slot = nullptr;
      for (auto& sl : S->slots)
        if (!sl.busy) {
          free_slot = &sl;
          break;
        }
      if (!free_slot) break;
      std::unique_ptr<Request> r;
      qw_status st = QW_OK;
      {
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->pending.empty()) break;
        if (!admit_memory(S, *S->pending.front(), *free_slot, &st)) break;
        r = std::move(S->pending.front());
        S->pending.pop_front();
        S->results[r->ticket].state = T_RUNNING;
        S->admitted++;
      }
      idle = false;
      free_slot->r = std::move(r);
      free_slot->busy = true;
      if (st == QW_OK) st = launch_request(S, *free_slot);
      if (st != QW_OK) {
        cudaStreamSynchronize(free_slot->stream);
        finish_slot(S, *free_slot, st);
      }
    }
    std::unique_lock<std::mutex> lock(S->mu);
    if (S->stop) {
      bool any = false;
      for (auto& sl : S->slots) any |= sl.busy;
      if (!any) break;
    }
    if (idle) S->cv.wait_for(lock, std::chrono::microseconds(50));
  }
}

}  // namespace qw

extern "C" {

qw_status qw_server_create(size_t hbm_budget_bytes, int slots, int max_pending, qw_server* out) {
  if (!out || hbm_budget_bytes < (size_t(1) << 20) || slots < 1 || slots > 64 || max_pending < 1) {
    set_error("qw_server_create: need out, budget >= 1 MiB, 1 <= slots <= 64, max_pending >= 1");
    return QW_EINVAL;
  }
  *out = nullptr;
  qw_server_s* S = new (std::nothrow) qw_server_s();
  if (!S) {
    set_error("qw_server_create: host allocation failed");
    return QW_ENOMEM;
  }
  S->budget = hbm_budget_bytes;
  S->max_pending = (size_t)max_pending;
  cudaError_t e = cudaGetDevice(&S->device);
  if (e == cudaSuccess) e = cudaMalloc(&S->pool_base, hbm_budget_bytes);
  S->pool.init(hbm_budget_bytes);
  S->slots.resize(slots);
  for (auto& sl : S->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&sl.d_res, 16 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&sl.d_part, 4 * kObsBlocks * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_res, 16 * sizeof(double));
  }
  if (e != cudaSuccess) {
    qw_status st = cuda_fail(e, "qw_server_create: allocation");
    qw_server_destroy(S);
    return st;
  }
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return QW_OK;
}

qw_status qw_submit(qw_server S, const qw_request* req, uint64_t* ticket) {
  if (!S || !req || !ticket) {
    set_error("qw_submit: null argument");
    return QW_EINVAL;
  }
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) {
    set_error("qw_submit: host allocation failed");
    return QW_ENOMEM;
  }
  r->req = *req;
  if (!make_geometry(req->dim, req->N, &r->g) || !(req->mass >= 0.0 && req->mass <= 1.0) || req->t < 0) {
    set_error("qw_submit: bad dim/N/mass/t");
    return QW_EINVAL;
  }
  if (!fft_size_ok(r->g.nx) || !fft_size_ok(r->g.ny) || !fft_size_ok(r->g.nz)) {
    set_error("qw_submit: the served (spectral) path needs 2^a 3^b axis lengths");
    return QW_EINVAL;
  }
  if (!req->psi0_host && !(req->sigma > 0.0)) {
    set_error("qw_submit: no field and no packet width");
    return QW_EINVAL;
  }
  // the box size's FFT tables (host-side planning only; nothing touches the GPU here)
  r->bytes_tables = fft_plan_table_bytes(r->g, QW_C64);
  const size_t need = request_bytes(r->g, &r->bytes_field, &r->bytes_omega) + 512 + ((r->bytes_tables + 255) & ~size_t(255));
  if (need > S->budget) {
    set_error("qw_submit: request needs %zu bytes, more than the server's HBM budget of %zu", need, S->budget);
    return QW_EINVAL;
  }
  if (req->psi0_host) {
    const unsigned char* p = static_cast<const unsigned char*>(req->psi0_host);
    r->psi0.assign(p, p + r->bytes_field);
    r->req.psi0_host = nullptr;
  }
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->pending.size() >= S->max_pending) {
      set_error("qw_submit: pending queue full (%zu)", S->max_pending);
      return QW_EAGAIN;
    }
    r->ticket = S->next_ticket++;
    *ticket = r->ticket;
    S->results[r->ticket] = Result();
    S->pending.push_back(std::move(r));
  }
  S->cv.notify_one();
  return QW_OK;
}

qw_status qw_poll(qw_server S, uint64_t ticket, qw_obs* out, int* done, double* latency_s) {
  if (!S || !done) {
    set_error("qw_poll: null argument");
    return QW_EINVAL;
  }
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->results.find(ticket);
  if (it == S->results.end()) {
    set_error("qw_poll: unknown ticket %llu", (unsigned long long)ticket);
    return QW_ENOTFOUND;
  }
  *done = 0;
  if (it->second.state == T_FAILED) {
    set_error("served request %llu failed: %s", (unsigned long long)ticket, it->second.error.c_str());
    *done = 1;
    S->results.erase(it);
    return QW_ECUDA;
  }
  if (it->second.state != T_DONE) return QW_OK;
  *done = 1;
  if (out) *out = it->second.obs;
  if (latency_s) *latency_s = it->second.latency;
  S->results.erase(it);
  return QW_OK;
}

qw_status qw_server_stats(qw_server S, qw_server_stats_t* out) {
  if (!S || !out) {
    set_error("qw_server_stats: null argument");
    return QW_EINVAL;
  }
  std::lock_guard<std::mutex> lock(S->mu);
  out->pending = (int64_t)S->pending.size();
  int busy = 0;
  for (auto& sl : S->slots) busy += sl.busy ? 1 : 0;
  out->running = busy;
  out->admitted = (int64_t)S->admitted;
  out->completed = (int64_t)S->completed;
  out->bytes_in_use = (int64_t)S->pool.used();
  out->peak_bytes = (int64_t)S->pool.peak();
  out->budget_bytes = (int64_t)S->budget;
  return QW_OK;
}

qw_status qw_server_destroy(qw_server S) {
  if (!S) return QW_OK;
  if (S->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lock(S->mu);
      S->stop = true;
      S->pending.clear();
    }
    S->cv.notify_one();
    S->worker.join();
  }
  cudaDeviceSynchronize();
  for (auto& sl : S->slots) {
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.d_res) cudaFree(sl.d_res);
    if (sl.d_part) cudaFree(sl.d_part);
    if (sl.h_res) cudaFreeHost(sl.h_res);
  }
  for (auto& kv : S->ffts) {
    fft_plan_destroy(&kv.second->plan);
    if (kv.second->ready) cudaEventDestroy(kv.second->ready);
  }
  if (S->pool_base) cudaFree(S->pool_base);
  delete S;
  return QW_OK;
}

}  // extern "C"
