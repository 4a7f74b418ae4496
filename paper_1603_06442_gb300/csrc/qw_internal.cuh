// Internal declarations shared by the translation units of libqw.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include <vector>

#include "qw.h"
#include "qw_fft.cuh"

namespace qw {

// ---- tracing: an NVTX range around each ABI call (header-only NVTX 3: free unless a
// profiler such as Nsight Systems attaches and records the ranges) ---------------------
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---- errors ---------------------------------------------------------------
void set_error(const char* fmt, ...);
qw_status cuda_fail(cudaError_t e, const char* what);

// Raise a kernel's dynamic shared-memory limit on the current device to at least `bytes`
// (per kernel and device the limit only grows).  Thread-safe: the server's scheduler
// thread and callers' threads launch the same kernels, possibly on different devices.
qw_status smem_attr_once(const void* func, int bytes);
template <typename K>
inline qw_status smem_attr(K* kernel, int bytes) {
  return smem_attr_once(reinterpret_cast<const void*>(kernel), bytes);
}
// Blocks of a kernel resident on the current device at once (0 if the query fails).
int resident_blocks_once(const void* func, int threads, int smem);
template <typename K>
inline int resident_blocks(K* kernel, int threads, int smem = 0) {
  return resident_blocks_once(reinterpret_cast<const void*>(kernel), threads, smem);
}

#define QW_CHECK_CUDA(call)                                        \
  do {                                                             \
    cudaError_t qw_e_ = (call);                                    \
    if (qw_e_ != cudaSuccess) return ::qw::cuda_fail(qw_e_, #call); \
  } while (0)

#define QW_CHECK_LAUNCH(what)                                      \
  do {                                                             \
    cudaError_t qw_e_ = cudaGetLastError();                        \
    if (qw_e_ != cudaSuccess) return ::qw::cuda_fail(qw_e_, what);  \
  } while (0)

template <typename T> struct CplxOf2;
template <> struct CplxOf2<float> { using t = float2; };
template <> struct CplxOf2<double> { using t = double2; };

// ---- debug poison (api.cu): while on, scratch and partner buffers are filled with NaN
// (all bytes 0xFF) before each call that must write them before reading them
bool debug_poison();
constexpr int kPoisonByte = 0xFF;  // 0xFFFFFFFF / 0xFFFF...FF are NaN in FP32 and FP64

// ---- autotune cache (api.cu) ------------------------------------------------
// A text file of "key | value" lines; the key starts with the GPU model.  Lookups take the
// last line with the key; stores append.  Both are no-ops while no cache file is set.
bool autotune_cache_get(const char* kind, const char* problem, std::vector<double>* values);
void autotune_cache_put(const char* kind, const char* problem, const std::vector<double>& values);

// ---- geometry -------------------------------------------------------------
// One field in the device layout: ncoset x s planes of `vol` complex values,
// each plane [z][y][x] with extents (nz, ny, nx).  1D: nx = N, ny = nz = 1;
// 2D: nx = ny = N; 3D (BCC): nx = ny = nz = M = N/2 and ncoset = 2.
struct Geometry {
  int dim;
  int64_t N;
  int s;
  int ncoset;
  int64_t nx, ny, nz;
  int64_t vol;    // nx * ny * nz
  int64_t elems;  // ncoset * s * vol
  int64_t sites;  // ncoset * vol
};

bool make_geometry(int dim, int64_t N, Geometry* g);

// Fields need only element alignment (8 bytes in complex64); kernels that move 16-byte
// vectors are chosen only for fields that are 16-byte aligned.
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Mass coefficients of one step.  With the Weyl sums S carrying the factor 4
// of the +-1 +- i entries, one output is  nq * S + i m * psi_other  with
// nq = n/4 (2D, 3D) or n (1D).  FP32 keeps nq and m as hi + lo pairs so that
// the fused multiply-adds use the FP64 values to ~2^-48 (no per-step bias).
struct Coef32 {
  float nq_hi, nq_lo, m_hi, m_lo;
};
struct Coef64 {
  double nq, m;
};
Coef32 make_coef32(int dim, double n, double m);
Coef64 make_coef64(int dim, double n, double m);

// ---- kernels (stencil.cu, stencil_tma.cu) ----------------------------------
// One update out = U in (Eq. upd-rule); in != out.  `variant` selects the
// kernel (qw_stencil_variant); QW_STENCIL_AUTO resolves to the best one that
// supports the geometry.
bool stencil_supported(const Geometry& g, qw_dtype dt, int variant);
qw_status launch_step(const Geometry& g, qw_dtype dt, int variant, double n, double m, const void* in, void* out,
                      cudaStream_t st);
bool tma_step_supported(const Geometry& g);
// Work items {tile, z_begin, z_end, 0} of the TMA stencils (tiles of 64 x ty cells)
// for `resident` CTAs.
std::vector<int4> tma_item_table(const Geometry& g, int resident, int ty);
bool tma2_step_supported(const Geometry& g);
// Two fused steps out = U^2 in (TMA, tiles of 64 x 8 cells).
qw_status launch_step_tma2(const Geometry& g, double n, double m, const void* in, void* out, const int4* items,
                           int nitems, int* err, int* next_item, cudaStream_t st);
qw_status launch_step_tma(const Geometry& g, double n, double m, const void* in, void* out, const int4* items,
                          int nitems, int* err, int* next_item, cudaStream_t st);
// FUSED: `steps` <= depth updates in one launch, box tiles of the field and a halo in shared
// memory (complex64, any geometry whose tile fits shared memory; batch.cu).
bool fused_step_supported(const Geometry& g, qw_dtype dt, int depth, const int* box);
qw_status launch_step_fused(const Geometry& g, int depth, const int* box, int steps, double n, double m,
                            const void* in, void* out, cudaStream_t st);

// ---- device reduction helpers ------------------------------------------------
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum NV doubles over a block of NT threads; thread 0 holds the totals.
template <int NV, int NT>
__device__ __forceinline__ void block_sum(double (&acc)[NV]) {
  __shared__ double sh[NT / 32][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = warp_sum_d(acc[j]);
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) sh[wid][j] = acc[j];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = warp_sum_d(lane < NT / 32 ? sh[lane][j] : 0.0);
  }
  __syncthreads();
}

// ---- reductions (observables.cu) -------------------------------------------
// Partial sums (norm, sum x|psi|^2, sum y|psi|^2, sum z|psi|^2) per block into
// `partials` (4 * kObsBlocks doubles), then one block folds them in a fixed
// order into `result` (4 doubles).  Deterministic for a given geometry.
constexpr int kObsBlocks = 608;  // 4 x 152 SMs
constexpr int kObsThreads = 256;
// Ten FP64 sums (n, S_x, S_y, S_z, S_xx, S_yy, S_zz, S_xy, S_xz, S_yz) of the density over
// the position coordinates into result; partials: 10 * kMom2MaxBlocks doubles.
constexpr int kMom2MaxBlocks = 4096;
qw_status launch_position_moments2(const Geometry& g, qw_dtype dt, const void* psi, double* partials,
                                   double* result, cudaStream_t st);
qw_status launch_position_moments(const Geometry& g, qw_dtype dt, const void* psi, double* partials,
                                  double* result, cudaStream_t st);
// K (2 or 4) sums over nblk partials [nblk][K] into result, in a fixed order; with many partials
// kFoldCtas CTAs fold ranges into stage (K * kFoldCtas doubles) first.
constexpr int kFoldCtas = 64;
qw_status launch_fold_partials(const double* partials, int64_t nblk, int K, double* stage, double* result,
                               cudaStream_t st);

// ---- spectral path (spectral.cu) ---------------------------------------------
struct SpecAxes {  // digit split of each axis (storage order -> frequency) and trig tables
  int nparts[3];
  int part[3][3];
  int64_t len[3];
  const double2* trig[3];
  const float2* trig32[3];
  const double2* angle;
  const float4* trigdf[3];
  const float4* angdf;
};
SpecAxes spec_axes(const Geometry& g, const FftPlan& f);
// omega per wave vector: (split = false, complex128 plans) a double-double (hi, lo) in 16
// bytes, or (split, complex64 plans) nu = omega / 2 pi as an FP32 (hi, lo) pair in 8 bytes
qw_status launch_omega_table(const Geometry& g, const SpecAxes& ax, double n, double m, double* omega,
                             cudaStream_t st, bool split);
// psi_hat (forward DFT, storage order) <- D_k^t psi_hat / |V|, BCC cosets mixed per cell;
// with norm0 (device, optional) the result is also divided by sqrt(norm0[0]);
// omega == nullptr computes omega_k in the kernel (FP64) instead of reading a table.
// Fused x pass: forward DFT along x, D_k^t, inverse DFT along x (complex64, 2D/BCC,
// x axis in one register pass); y and z are transformed around it by the caller.
bool fused_x_supported(const Geometry& g, const FftPlan& f, qw_dtype dt);
qw_status launch_evolve_fused_x(const Geometry& g, const SpecAxes& ax, const FftPlan& f, double n, double m,
                                const double* omega, int64_t t, void* psi, cudaStream_t st,
                                const double* norm0 = nullptr);
// With the same tiling, the particle-weight sums of a spectrum still to be transformed
// along x (complex64): 2 doubles per CTA (fused_x_grid CTAs) into partials, folded into
// result[0..1] through the 2 * kFoldCtas doubles after them; data is only read.
int64_t fused_x_grid(const Geometry& g);
qw_status launch_weights_fused_x(const Geometry& g, const SpecAxes& ax, const FftPlan& f, double n, double m,
                                 const void* data, double* partials, double* result, cudaStream_t st);
// Per-wave-vector Foldy-Wouthuysen coefficients of a forward spectrum, in place (with the
// inverse transform's 1/|V| scale folded in).
qw_status launch_fw_pointwise(const Geometry& g, const SpecAxes& ax, qw_dtype dt, double n, double m, void* psi_hat,
                              cudaStream_t st);
qw_status launch_evolve_pointwise(const Geometry& g, const SpecAxes& ax, qw_dtype dt, double n, double m,
                                  const double* omega, int64_t t, void* psi_hat, cudaStream_t st,
                                  const double* norm0 = nullptr);

// ---- state preparation (packet.cu) ---------------------------------------------
// psi(x) = exp(-|d|^2 / (4 sigma^2)) exp(i k0.d) chi with d the minimum-image
// displacement from x0 on the periodic box (physical BCC coordinates, lattice
// coordinates in 2D); chi = s complex values (re, im interleaved).  Not normalised.
qw_status launch_packet(const Geometry& g, qw_dtype dt, const double* x0, double sigma, const double* k0,
                        const double* chi, void* psi, cudaStream_t st);
// (sum |psi^|^2, sum psi^dag G/sin(omega) psi^) over the zone into result[0..1].
// ---- probability projections (projection.cu) ---------------------------------
// keep: bit 0 x, bit 1 y, bit 2 z.  projection_partials: doubles of chunk partials the
// launch needs (0: none); projection_outputs: N^(kept axes).
int64_t projection_partials(const Geometry& g, int keep, qw_dtype dt);
int64_t projection_outputs(const Geometry& g, int keep);
qw_status launch_projection(const Geometry& g, qw_dtype dt, const void* psi, int keep, double* out,
                            double* partials, cudaStream_t st);

qw_status launch_particle_weights(const Geometry& g, const SpecAxes& ax, qw_dtype dt, double n, double m,
                                  const void* psi_hat, double* partials, double* result, cudaStream_t st);

}  // namespace qw

// ---- the plan ---------------------------------------------------------------
// Device fields of a host-field run: field j lives in buffer j % kHostBufs, so a field's copy
// can start two steps before its step (a slow transfer has two steps to finish).
constexpr int kHostBufs = 3;

struct qw_plan_s {
  qw::Geometry g;
  double mass;
  double n;
  qw_dtype dtype;
  int device;
  size_t elem_bytes;
  int stencil;          // qw_stencil_variant in use (never AUTO after creation)
  int fuse_depth;       // FUSED variant: steps per launch and tile box (x, y, z cells)
  int fuse_box[3];
  void* scratch;        // one field: ping-pong partner of the caller's buffer
  int* dev_flags;       // [0] error word of bounded device waits, [1] work counter
  int4* tma_items;      // work-item table of the TMA stencil (device), or null
  int tma_nitems;
  int4* tma2_items;     // work-item table of the two-step TMA stencil, or null
  int tma2_nitems;
  // spectral path (allocated by the first spectral call or qw_plan_prepare_spectral)
  bool spec_ready;
  qw::FftPlan fft;
  double* omega;        // omega_k per stored wave vector (BCC: q0 of each cell): a double-double
                        // (16 B) for complex128, nu = omega / 2 pi as an FP32 pair (8 B) for complex64
  double* spec_partials;  // 2 * kObsBlocks doubles for the particle-weight reduction
  double* xw_partials;    // 2 doubles per CTA of the x-pass weights (when the x pass is fused), then
                          // 2 * kFoldCtas for the fold's first stage
  double* zm_partials;    // 4 doubles per CTA of the first forward pass of the observables, when it
  int64_t zm_ctas;        // takes the norm and <x> of the field it reads (0: a separate kernel does),
                          // then 4 * kFoldCtas for the fold's first stage
  double* red_partials; // 10 * kMom2MaxBlocks doubles (>= 4 * kObsBlocks)
  double* red_result;   // 16 doubles (device)
  double* red_host;     // 16 doubles (pinned host); the last holds the copied error word
  // host-field runs (qw_run_host): kHostBufs device fields, a copy stream and its events,
  // allocated by the first call
  void* hbuf[kHostBufs];
  cudaStream_t copy_stream;
  cudaEvent_t ev_copied[kHostBufs], ev_freed[kHostBufs], ev_stepped[kHostBufs];
  double* hstage;  // 2 x 8 doubles (pinned): observables of the two fields in flight
  // optional per-field timing of qw_run_host: for field j, events (timing enabled) at its copy's
  // start and end (copy stream) and at its step's start and end and its observables' end
  // (compute stream); tev_fields = fields recorded by the last run
  bool host_timing;
  std::vector<cudaEvent_t> tev;
  int tev_fields;
  // probability projections: chunk partials, grown on demand
  double* proj_partials;
  int64_t proj_cap;
};
