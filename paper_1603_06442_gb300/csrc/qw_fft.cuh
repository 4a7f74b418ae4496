// FFT plan types of the spectral path (fft.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qw.h"

namespace qw {

struct Geometry;

constexpr int kMaxStages = 16;
constexpr int kFftSmemBytes = 131072;   // two ping-pong tiles
constexpr int kMaxLineF32 = 8192;       // longest single-pass line (complex64)
constexpr int kMaxLineF64 = 4096;       // (complex128)

// One in-place pass: DFTs of length L over elements o*(L*S) + j*S + i.
struct FftPass {
  int L;
  int64_t S;
  int64_t O;
  int C;            // lines per CTA (a power of two)
  int cshift;       // log2(C)
  int pitch;        // shared-memory line pitch (elements)
  size_t smem;      // dynamic shared memory bytes
  int nstages;
  int radix[kMaxStages];
  int twiddle;      // apply exp(-+2 pi i k (i / tw_div) / tw_N) after (forward) / before (inverse)
  int64_t tw_N;
  int64_t tw_div;
  int tlo_bits;
  void* tw_line = nullptr;  // exp(-2 pi i m / L), m < L
  void* tw_hi = nullptr;    // two-level table of exp(-2 pi i m / tw_N)
  void* tw_lo = nullptr;
};

// Position moments taken by the out-of-place first pass of an axis while it holds its
// source in shared memory (observables): per CTA the FP64 sums (n, sum X d, sum Y d,
// sum Z d), d = |psi_q(x)|^2 of the CTA's lines, X physical (BCC: 2 m + c).
struct FftMoments {
  int dim;
  int nx;
  int s;              // spinor components per coset
  double* partials;   // 4 doubles per CTA
};

struct FftAxis {
  int nparts;       // 1..3 digits of the axis length
  int part[3];
  int first;        // index of the first pass
  int count;
};

struct FftPlan {
  qw_dtype dtype = QW_C64;
  int npass = 0;
  FftPass pass[9];
  FftAxis axis[3];
  // (cos, sin) tables of the symbol's angles, FP64 (double2), per axis:
  //   dim 1: 2 pi f / N (f < N);  dim 2: pi q / N (q < 2N, for k1 +- k2 halves);
  //   dim 3: pi f / M (f < M, the half wave vector kappa / 2 of each axis)
  void* trig[3] = {nullptr, nullptr, nullptr};
  void* trig32[3] = {nullptr, nullptr, nullptr};  // the same tables as float2 (complex64 kernels)
  // (cos, sin)(j * kAngleStep), j <= kAngleTab: anchors of the fast omega_k refinement
  void* angle = nullptr;
  // double-float copies (float4: cos hi, cos lo, sin hi, sin lo) of the symbol tables and
  // the anchors, for the FP64-free omega_k of complex64 requests.  The chain (dim 1)
  // uses two levels instead of a table as long as the chain: angle 2 pi (kDfFine q1 + q0) / N
  // from trigdf[1][q1] (coarse) and trigdf[0][q0] (fine).
  void* trigdf[3] = {nullptr, nullptr, nullptr};
  void* angdf = nullptr;
  bool external_tables = false;  // tables carved from a caller's region (not freed here)
  size_t field_bytes = 0;        // one field (an axis of length 1 has no pass: an out-of-place
                                 // transform along it is a copy)
};

// Destination of a plan's tables when they are not cudaMalloc'd: a region of device
// memory owned by the caller, filled in order on `st` by a table kernel (no allocation,
// no host work, asynchronous).  base == nullptr counts the bytes only.
struct TableDst {
  char* base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  cudaStream_t st = nullptr;
};

constexpr int kDfFine = 4096;

constexpr int kAngleTab = 1024;
constexpr double kAngleStep = 3.14159265358979323846 / kAngleTab;

bool fft_size_ok(int64_t L);
// dst == nullptr: tables cudaMalloc'd and computed on the host (synchronous).
qw_status fft_plan_create(FftPlan* f, const Geometry& g, qw_dtype dt, TableDst* dst = nullptr);
// Device bytes of a plan's tables in a TableDst region (0 if the geometry has no plan).
size_t fft_plan_table_bytes(const Geometry& g, qw_dtype dt);
void fft_plan_destroy(FftPlan* f);
// Forward over all axes (x, then y, then z) / inverse (z, y, x); unnormalised.
qw_status fft_forward(const FftPlan& f, int dim, void* data, cudaStream_t st);
qw_status fft_inverse(const FftPlan& f, int dim, void* data, cudaStream_t st);
qw_status fft_forward_axis(const FftPlan& f, int ax, void* data, cudaStream_t st);
qw_status fft_inverse_axis(const FftPlan& f, int ax, void* data, cudaStream_t st);
// Forward passes of one axis reading src and writing dst (the first pass out of place,
// the rest in place on dst); src is not modified.
qw_status fft_forward_axis_from(const FftPlan& f, int ax, const void* src, void* dst, cudaStream_t st);
// CTAs of the moments-taking form of fft_forward_axis_from along axis ax: 0 when it has none
// (complex64 axes transformed in one register pass with a stride, i.e. not the x axis).
int64_t fft_moment_ctas(const FftPlan& f, int ax);
// fft_forward_axis_from that also writes the position moments of src (FftMoments) into
// m.partials, fft_moment_ctas(f, ax) CTAs of four doubles; QW_EINVAL where that is 0.
qw_status fft_forward_axis_from_moments(const FftPlan& f, int ax, const void* src, void* dst, const FftMoments& m,
                                        cudaStream_t st);

}  // namespace qw
