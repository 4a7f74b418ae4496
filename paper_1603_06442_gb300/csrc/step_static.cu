// qw_step_static: the stencil stepping of qw_step without any device allocation.
//
// qw_step ping-pongs between the caller's field and a scratch field that
// qw_plan_create allocates.  Some callers cannot allocate device memory at the
// point where they step a walk: code whose device memory is owned and budgeted
// by another allocator (a framework's caching pool that already holds the
// GPU), or a latency-critical loop where cudaMalloc's implicit device-wide
// synchronisation is not acceptable.  For them the ping-pong partner lives in
// the file-scope array below, which every GPU that loads this library holds
// until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "qw_internal.cuh"

namespace qw {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_step_scratch[kStaticScratchBytes];

// Device address of g_step_scratch, looked up once per device with that device
// current (in host code the symbol name is only a host-side stand-in).
static void* g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mu;

static qw_status static_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("qw_step_static: device ordinal %d out of range", dev);
    return QW_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_step_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "qw_step_static: cudaGetSymbolAddress");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return QW_OK;
}

}  // namespace qw

using namespace qw;

extern "C" qw_status qw_step_static(int dim, int64_t N, double mass, qw_dtype dtype, void* psi, int64_t nsteps,
                                    void* stream) {
  NvtxRange nvtx_range("qw_step_static");
  Geometry g;
  if (!make_geometry(dim, N, &g)) {
    set_error("qw_step_static: bad dim=%d / N=%lld", dim, (long long)N);
    return QW_EINVAL;
  }
  if (!(mass >= 0.0 && mass <= 1.0) || (dtype != QW_C64 && dtype != QW_C128) || !psi || nsteps < 0) {
    set_error("qw_step_static: bad mass, dtype, field pointer or step count");
    return QW_EINVAL;
  }
  const size_t bytes = (size_t)g.elems * (dtype == QW_C64 ? 8 : 16);
  if (bytes > kStaticScratchBytes) {
    set_error("qw_step_static: the field needs %zu bytes of scratch, more than the %zu-byte static maximum "
              "(use qw_plan_create + qw_step for larger fields)",
              bytes, kStaticScratchBytes);
    return QW_EINVAL;
  }
  if (nsteps == 0) return QW_OK;
  int dev = 0;
  QW_CHECK_CUDA(cudaGetDevice(&dev));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the scratch address below belongs to the current device: the stream must too
  int sdev = -1;
  QW_CHECK_CUDA(cudaStreamGetDevice(s, &sdev));
  if (sdev != dev) {
    set_error("qw_step_static: the stream belongs to device %d but device %d is current; make the field's "
              "and the stream's device current first",
              sdev, dev);
    return QW_EINVAL;
  }
  void* scratch = nullptr;
  qw_status st = static_scratch(dev, &scratch);
  if (st != QW_OK) return st;
  // VEC moves 16-byte vectors: only for 16-byte aligned fields (the scratch array is)
  const int variant =
      (stencil_supported(g, dtype, QW_STENCIL_VEC) && aligned16(psi)) ? QW_STENCIL_VEC : QW_STENCIL_PLAIN;
  const double n = std::sqrt(1.0 - mass * mass);
  if (debug_poison()) QW_CHECK_CUDA(cudaMemsetAsync(scratch, kPoisonByte, bytes, s));
  void* cur = psi;
  void* nxt = scratch;
  for (int64_t i = 0; i < nsteps; ++i) {
    st = launch_step(g, dtype, variant, n, mass, cur, nxt, s);
    if (st != QW_OK) return st;
    void* t = cur;
    cur = nxt;
    nxt = t;
  }
  if (cur != psi) QW_CHECK_CUDA(cudaMemcpyAsync(psi, cur, bytes, cudaMemcpyDeviceToDevice, s));
  return QW_OK;
}
