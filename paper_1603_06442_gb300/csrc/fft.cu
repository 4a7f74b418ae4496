// Batched in-place DFT passes along one axis of the device layout (the Fourier
// form of Sec. 4 needs forward and inverse DFTs of every component plane; the
// paper names the Cooley-Tukey FFT, this is a mixed-radix Stockham variant).
//
// Conventions: forward X[k] = sum_n x[n] exp(-2 pi i k n / L), inverse with
// exp(+...) and no normalisation (the pointwise step applies 1/|V|).
//
// One pass transforms lines of length L <= kMaxLine whose elements sit at
//     o * (L * S) + j * S + i          (o < O outer, j < L, i < S inner),
// CTA tiles of C lines x L elements live in shared memory (ping-pong buffers,
// line-minor with an odd pitch so both load patterns are conflict-free), and
// every stage is a radix-R butterfly (R in 8, 4, 3, 2) of the Stockham
// autosort recursion: natural order in, natural order out.
//
// Axes longer than kMaxLine are split L = A * B (Cooley-Tukey index map):
// a pass of length A with stride B (followed by the twiddle
// exp(-2 pi i k b / L)) and a pass of length B on contiguous segments.  The
// spectrum is then left in the digit-permuted order position B k1 + k2 <->
// frequency k1 + A k2, which the pointwise kernels decode; the inverse undoes
// the passes in reverse order, so fields return in natural order.
#include <cuda_runtime.h>

#include <cmath>
#include <algorithm>
#include <type_traits>
#include <vector>

#include "qw_fft.cuh"
#include "qw_internal.cuh"
#include "qw_regdft.cuh"

namespace qw {

template <typename T, bool INV>
__global__ void __launch_bounds__(256) fft_pass_kernel(typename Cx<T>::t* __restrict__ data, FftPass p,
                                                       const typename Cx<T>::t* __restrict__ tw_line,
                                                       const typename Cx<T>::t* __restrict__ tw_hi,
                                                       const typename Cx<T>::t* __restrict__ tw_lo) {
  using V = typename Cx<T>::t;
  extern __shared__ __align__(16) unsigned char fft_smem[];
  V* bufA = reinterpret_cast<V*>(fft_smem);
  V* bufB = bufA + (size_t)p.L * p.pitch;
  const int L = p.L, C = p.C, pitch = p.pitch;
  const int64_t S = p.S;
  const int64_t nlines = p.O * S;
  const int64_t l0 = (int64_t)blockIdx.x * C;
  const int ncol = (int)((nlines - l0) < C ? (nlines - l0) : C);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int total = L * ncol;

  // ---- load (and undo the inter-pass twiddle on the inverse) ----
  // C divides the block, so for S > 1 every thread keeps one column c and its
  // line base; for S == 1 the CTA's lines are one contiguous run.
  const int cfix = tid % C;
  int64_t base_c = 0, twb_c = 0;
  {
    const int64_t l = l0 + cfix;
    if (l < nlines) {
      const int64_t o = l / S, i = l - o * S;
      base_c = o * (int64_t)L * S + i;
      twb_c = i / p.tw_div;
    }
  }
  if (S == 1) {
    for (int e = tid; e < total; e += nthr) {
      const int c = e / L, j = e - c * L;
      bufA[j * pitch + c] = data[l0 * L + e];
    }
  } else if (cfix < ncol) {
    for (int j = tid / C; j < L; j += nthr / C) {
      V v = data[base_c + (int64_t)j * S];
      if (INV && p.twiddle) v = cmulc(v, twiddle_big(tw_hi, tw_lo, (int64_t)j * twb_c, p.tlo_bits));
      bufA[j * pitch + cfix] = v;
    }
  }
  __syncthreads();

  // ---- Stockham stages ----
  V* in = bufA;
  V* out = bufB;
  int Ns = 1;
  for (int s = 0; s < p.nstages; ++s) {
    const int R = p.radix[s];
    const int nb = L / R;
    const int tstep = L / (Ns * R);  // table stride of omega_{Ns R}
    // butterfly b = tid + i * nthr: column c is fixed, jb advances by nthr / C;
    // k = jb % Ns and jq = jb / Ns advance by precomputed quotient/remainder
    const int jstep = nthr >> p.cshift;
    const int sq = jstep / Ns, sr = jstep - sq * Ns;
    const int c = tid & (C - 1);
    int jb = tid >> p.cshift;
    int jq = jb / Ns, k = jb - jq * Ns;
    for (; jb < nb; jb += jstep) {
      if (c < ncol) {
      const int idxD = jq * Ns * R + k;
      if (R == 8) {
        V a[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          a[r] = in[(jb + r * nb) * pitch + c];
          if (r > 0 && Ns > 1) {
            const V w = tw_line[r * k * tstep];
            a[r] = INV ? cmulc(a[r], w) : cmul(a[r], w);
          }
        }
        dft8<INV, T>(a);
#pragma unroll
        for (int r = 0; r < 8; ++r) out[(idxD + r * Ns) * pitch + c] = a[r];
      } else if (R == 4) {
        V a[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          a[r] = in[(jb + r * nb) * pitch + c];
          if (r > 0 && Ns > 1) {
            const V w = tw_line[r * k * tstep];
            a[r] = INV ? cmulc(a[r], w) : cmul(a[r], w);
          }
        }
        dft4<INV>(a[0], a[1], a[2], a[3]);
#pragma unroll
        for (int r = 0; r < 4; ++r) out[(idxD + r * Ns) * pitch + c] = a[r];
      } else if (R == 3) {
        V a[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          a[r] = in[(jb + r * nb) * pitch + c];
          if (r > 0 && Ns > 1) {
            const V w = tw_line[r * k * tstep];
            a[r] = INV ? cmulc(a[r], w) : cmul(a[r], w);
          }
        }
        dft3<INV, T>(a[0], a[1], a[2]);
#pragma unroll
        for (int r = 0; r < 3; ++r) out[(idxD + r * Ns) * pitch + c] = a[r];
      } else {
        V a0 = in[jb * pitch + c], a1 = in[(jb + nb) * pitch + c];
        if (Ns > 1) {
          const V w = tw_line[k * tstep];
          a1 = INV ? cmulc(a1, w) : cmul(a1, w);
        }
        dft2<INV>(a0, a1);
        out[idxD * pitch + c] = a0;
        out[(idxD + Ns) * pitch + c] = a1;
      }
      }
      k += sr;
      jq += sq;
      if (k >= Ns) {
        k -= Ns;
        ++jq;
      }
    }
    __syncthreads();
    V* t = in;
    in = out;
    out = t;
    Ns *= R;
  }

  // ---- store (apply the inter-pass twiddle on the forward) ----
  if (S == 1) {
    for (int e = tid; e < total; e += nthr) {
      const int c = e / L, j = e - c * L;
      data[l0 * L + e] = in[j * pitch + c];
    }
  } else if (cfix < ncol) {
    for (int j = tid / C; j < L; j += nthr / C) {
      V v = in[j * pitch + cfix];
      if (!INV && p.twiddle) v = cmul(v, twiddle_big(tw_hi, tw_lo, (int64_t)j * twb_c, p.tlo_bits));
      data[base_c + (int64_t)j * S] = v;
    }
  }
}

// MOM (forward strided passes of the observables): the position moments of the loaded lines
// (FftMoments) are summed before the transform, one partial per CTA.
template <typename T, bool INV, int R1, int R2, bool CONTIG, bool MOM = false>
__global__ void __launch_bounds__(256) fft2f_kernel(typename Cx<T>::t* data, const typename Cx<T>::t* src, FftPass p,
                                                    const typename Cx<T>::t* __restrict__ tw_line,
                                                    const typename Cx<T>::t* __restrict__ tw_hi,
                                                    const typename Cx<T>::t* __restrict__ tw_lo,
                                                    FftMoments mom = FftMoments{}) {
  using V = typename Cx<T>::t;
  constexpr int L = R1 * R2;
  constexpr int TPL = R1 > R2 ? R1 : R2;  // threads per line
  constexpr int C = 256 / TPL;            // lines per CTA (C * TPL <= 256 threads work)
  constexpr int CP = (C % 2 == 0) ? C + 1 : C;  // odd line-minor pitch
  extern __shared__ __align__(16) unsigned char f2_smem[];
  V* sm = reinterpret_cast<V*>(f2_smem);
  const int tid = threadIdx.x;
  const int64_t S = p.S;
  const int64_t nlines = p.O * S;
  const int64_t l0 = (int64_t)blockIdx.x * C;
  const int c = tid % C, r = tid / C;   // r >= TPL: idle in the butterfly steps
  const int64_t l = l0 + c;
  const bool live = l < nlines && r < TPL;
  int64_t base = 0, tw_b = 0;
  if (live) {
    const int64_t o = l / S, i = l - o * S;
    base = o * (int64_t)L * S + i;
    tw_b = i / p.tw_div;
  }
  // twiddles of step A, read from the per-line table (L1-resident) when needed
  const TwRow<V> tw{tw_line, r};
  // ---- load into shared memory, element n of line c at sm[c + CP n], by cp.async: the
  // copies go straight to shared memory, so all of them are in flight at once without
  // holding registers (zero-filled past the last line)
  if (CONTIG) {  // S == 1: the CTA's lines are one contiguous run (never a twiddled pass)
    // element e = tid + 256 j of the run sits at line e / L, position e % L; both come
    // from tid / L and tid % L plus compile-time offsets (no division per element)
    constexpr int NE = (C * L + 255) / 256;
    const int t_c = tid / L, t_x = tid - (tid / L) * L;
#pragma unroll
    for (int j = 0; j < NE; ++j) {
      int xx = t_x + (256 * j) % L, cc = t_c + (256 * j) / L;
      if (xx >= L) {
        xx -= L;
        ++cc;
      }
      const bool ok = l0 + cc < nlines;
      if (cc < C) cp_async_elem(&sm[cc + CP * xx], ok ? src + l0 * L + tid + 256 * j : src, ok);
    }
    cp_async_wait_all();
  } else if (r < TPL) {
    constexpr int NL = (L + TPL - 1) / TPL;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const int n = r + TPL * j;
      if (n < L) cp_async_elem(&sm[c + CP * n], live ? src + base + (int64_t)n * S : src, live);
    }
    cp_async_wait_all();
    if (INV && p.twiddle && live) {  // the inverse applies the inter-pass twiddle on load
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        const int n = r + TPL * j;
        if (n < L) sm[c + CP * n] = cmulc(sm[c + CP * n], twiddle_big(tw_hi, tw_lo, (int64_t)n * tw_b, p.tlo_bits));
      }
    }
  }
  __syncthreads();
  __shared__ float mom_wsum[MOM ? 8 : 1][4];  // MOM: the warp sums, combined after the transform
  if constexpr (MOM) {
    // this thread's elements n = r + TPL j of line l: |v|^2 and the four sums in FP32 (the axis
    // coordinate from the local index j), FP32 warp sums, the CTA's eight warp sums in FP64 (an
    // FP64 operation costs ~64 FP32 ones here)
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    if (live) {
      constexpr int NL = (L + TPL - 1) / TPL;
      float g0 = 0.f, g1 = 0.f;
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        const int n = r + TPL * j;
        if (n < L) {
          const V v = sm[c + CP * n];
          const float d = v.x * v.x + v.y * v.y;
          g0 += d;
          g1 = fmaf((float)j, d, g1);
        }
      }
      const int o = (int)(l / S), i = (int)(l - (int64_t)o * S);  // plane (coset * s + component), position
      const float an = fmaf((float)r, g0, (float)TPL * g1);          // sum n d
      a[0] = g0;
      if (mom.dim == 3) {
        const float off = (float)(o / mom.s);
        a[1] = (2.f * (float)(i % mom.nx) + off) * g0;
        a[2] = (2.f * (float)(i / mom.nx) + off) * g0;
        a[3] = fmaf(2.f, an, off * g0);
      } else {  // 2D: lines along y at x = i
        a[1] = (float)i * g0;
        a[2] = an;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int w = 16; w > 0; w >>= 1) a[q] += __shfl_xor_sync(0xffffffffu, a[q], w);
    if ((tid & 31) == 0) {
#pragma unroll
      for (int q = 0; q < 4; ++q) mom_wsum[tid >> 5][q] = a[q];
    }
  }
  reg_fft_steps<T, INV, R1, R2, CP>(sm, c, r, tw);
  if constexpr (MOM) {  // the transform's barriers have published the warp sums
    if (tid == 0) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        double acc = 0.0;
        for (int w = 0; w < 8; ++w) acc += (double)mom_wsum[w][q];
        mom.partials[(int64_t)blockIdx.x * 4 + q] = acc;
      }
    }
  }
  // ---- store
  if (CONTIG) {
    constexpr int NE = (C * L + 255) / 256;
    const int t_c = tid / L, t_x = tid - (tid / L) * L;
#pragma unroll
    for (int j = 0; j < NE; ++j) {
      int xx = t_x + (256 * j) % L, cc = t_c + (256 * j) / L;
      if (xx >= L) {
        xx -= L;
        ++cc;
      }
      if (cc < C && l0 + cc < nlines) data[l0 * L + tid + 256 * j] = sm[cc + CP * xx];
    }
  } else if (r < TPL) {
#pragma unroll 4
    for (int n = r; n < L; n += TPL) {
      if (!live) break;
      V v = sm[c + CP * n];
      if (!INV && p.twiddle) v = cmul(v, twiddle_big(tw_hi, tw_lo, (int64_t)n * tw_b, p.tlo_bits));
      data[base + (int64_t)n * S] = v;
    }
  }
}

template <typename T, bool INV, int R1, int R2>
static qw_status launch_2f(const FftPass& p, void* data, const void* src, cudaStream_t st) {
  using V = typename Cx<T>::t;
  constexpr int L = R1 * R2, TPL = R1 > R2 ? R1 : R2, C = 256 / TPL;
  const size_t smem = (size_t)L * ((C % 2 == 0) ? C + 1 : C) * sizeof(V);
  const int64_t nlines = p.O * p.S;
  const int64_t grid = (nlines + C - 1) / C;
  if (grid > 0x7fffffff) {
    set_error("FFT grid too large");
    return QW_EINVAL;
  }
  if (p.S == 1) {
    const qw_status sa = smem_attr(fft2f_kernel<T, INV, R1, R2, true>, (int)smem);
    if (sa != QW_OK) return sa;
    fft2f_kernel<T, INV, R1, R2, true><<<(unsigned)grid, 256, smem, st>>>(
        static_cast<V*>(data), static_cast<const V*>(src), p, static_cast<const V*>(p.tw_line), static_cast<const V*>(p.tw_hi),
        static_cast<const V*>(p.tw_lo));
  } else {
    const qw_status sa = smem_attr(fft2f_kernel<T, INV, R1, R2, false>, (int)smem);
    if (sa != QW_OK) return sa;
    fft2f_kernel<T, INV, R1, R2, false><<<(unsigned)grid, 256, smem, st>>>(
        static_cast<V*>(data), static_cast<const V*>(src), p, static_cast<const V*>(p.tw_line), static_cast<const V*>(p.tw_hi),
        static_cast<const V*>(p.tw_lo));
  }
  QW_CHECK_LAUNCH("fft two-factor pass launch");
  return QW_OK;
}

// f(R1, R2) (as integral constants) for a register length L >= 64; false for other lengths.
template <typename F>
static bool with_reg_factors64(int L, F&& f) {
  switch (L) {
#define QW_2FF(LEN, A, B)                                                           \
  case LEN:                                                                         \
    if constexpr (LEN >= 64) {                                                      \
      f(std::integral_constant<int, A>{}, std::integral_constant<int, B>{});        \
      return true;                                                                  \
    }                                                                               \
    return false;
    QW_REG_LENGTHS_POW2(QW_2FF)
    QW_REG_LENGTHS_F32(QW_2FF)
#undef QW_2FF
    default:
      return false;
  }
}

// The moments-taking pass is a forward, untwiddled, strided complex64 register pass.
static bool moment_pass_ok(const FftPlan& f, int ax) {
  if (f.dtype != QW_C64 || ax < 0 || ax > 2) return false;
  const FftAxis& A = f.axis[ax];
  if (A.count != 1) return false;
  const FftPass& p = f.pass[A.first];
  return p.S > 1 && !p.twiddle && with_reg_factors64(p.L, [](auto, auto) {});
}

int64_t fft_moment_ctas(const FftPlan& f, int ax) {
  if (!moment_pass_ok(f, ax)) return 0;
  const FftPass& p = f.pass[f.axis[ax].first];
  int64_t ctas = 0;
  with_reg_factors64(p.L, [&](auto a, auto b) {
    constexpr int TPL = decltype(a)::value > decltype(b)::value ? decltype(a)::value : decltype(b)::value;
    constexpr int C = 256 / TPL;
    ctas = (p.O * p.S + C - 1) / C;
  });
  return ctas;
}

qw_status fft_forward_axis_from_moments(const FftPlan& f, int ax, const void* src, void* dst, const FftMoments& m,
                                        cudaStream_t st) {
  if (!moment_pass_ok(f, ax)) {
    set_error("moments pass: axis %d is not a single strided complex64 register pass", ax);
    return QW_EINVAL;
  }
  const FftPass& p = f.pass[f.axis[ax].first];
  qw_status out = QW_OK;
  with_reg_factors64(p.L, [&](auto a, auto b) {
    constexpr int R1 = decltype(a)::value, R2 = decltype(b)::value;
    constexpr int L = R1 * R2, TPL = R1 > R2 ? R1 : R2, C = 256 / TPL;
    const size_t smem = (size_t)L * ((C % 2 == 0) ? C + 1 : C) * sizeof(float2);
    const int64_t grid = (p.O * p.S + C - 1) / C;
    out = smem_attr(fft2f_kernel<float, false, R1, R2, false, true>, (int)smem);
    if (out != QW_OK) return;
    fft2f_kernel<float, false, R1, R2, false, true><<<(unsigned)grid, 256, smem, st>>>(
        static_cast<float2*>(dst), static_cast<const float2*>(src), p, static_cast<const float2*>(p.tw_line),
        static_cast<const float2*>(p.tw_hi), static_cast<const float2*>(p.tw_lo), m);
    const cudaError_t e = cudaGetLastError();
    out = e == cudaSuccess ? QW_OK : cuda_fail(e, "fft moments pass launch");
  });
  return out;
}

// Lengths with a two-factor register kernel; returns false for the generic path.
// With p == nullptr nothing is launched: the call only reports whether L has one
// (the planner uses this to split long axes into register-kernel passes).
#define QW_2F(LEN, A, B)                                 \
  case LEN:                                              \
    if (p) *out = launch_2f<T, INV, A, B>(*p, data, src, st); \
    return true;
template <typename T, bool INV>
static bool run_2f(int L, const FftPass* p, void* data, const void* src, cudaStream_t st, qw_status* out) {
  switch (L) {
    QW_REG_LENGTHS_POW2(QW_2F)
    default: break;
  }
  if (sizeof(T) != 4) return false;
  // lengths with a factor 3 (complex64; complex128 uses the Stockham kernel)
  switch (L) {
    QW_REG_LENGTHS_F32(QW_2F)
    default: return false;
  }
}
#undef QW_2F

// ---------------------------------------------------------------- planning
static bool radix_plan(int L, int* radix, int* n) {
  int k = 0;
  int r = L;
  while (r % 8 == 0 && r > 0) { radix[k++] = 8; r /= 8; }
  while (r % 4 == 0 && r > 0) { radix[k++] = 4; r /= 4; }
  while (r % 2 == 0 && r > 0) { radix[k++] = 2; r /= 2; }
  while (r % 3 == 0 && r > 0) { radix[k++] = 3; r /= 3; }
  if (r != 1 || k > kMaxStages) return false;
  *n = k;
  return true;
}

bool fft_size_ok(int64_t L) {
  if (L < 1) return false;
  while (L % 2 == 0) L /= 2;
  while (L % 3 == 0) L /= 3;
  return L == 1;
}

// Relative cost of one pass of length L: every pass reads and writes the whole
// field once; the generic shared-memory kernel runs several times slower than a
// register kernel (measured: ~0.7 against ~4 TB/s), worse still for short lines.
template <typename T>
static double pass_cost(int64_t L) {
  qw_status unused;
  if (run_2f<T, false>((int)L, nullptr, nullptr, nullptr, nullptr, &unused)) return 1.0;
  return L < 64 ? 8.0 : 4.0;
}

// Split an axis of length L (2^a 3^b) into 1-3 pass lengths <= maxline of least
// total cost; ties go to the most even split.
template <typename T>
static bool split_axis(int64_t L, int maxline, std::vector<int>* parts) {
  parts->clear();
  std::vector<int64_t> dv;  // divisors of L that can be one pass
  for (int64_t a = 1; a <= maxline; a *= 2)
    for (int64_t b = a; b <= maxline; b *= 3)
      if (b >= 2 && L % b == 0) dv.push_back(b);
  double best = 1e300;
  auto consider = [&](std::initializer_list<int64_t> fs) {
    double c = 0.0, spread = 0.0;
    int64_t lo = L, hi = 1;
    for (int64_t f : fs) {
      if (f < 2 || f > maxline) return;
      c += pass_cost<T>(f);
      lo = f < lo ? f : lo;
      hi = f > hi ? f : hi;
    }
    spread = 1e-9 * (double)(hi - lo);
    if (c + spread < best) {
      best = c + spread;
      parts->assign(fs.begin(), fs.end());
    }
  };
  if (L <= maxline) consider({L});
  for (int64_t d1 : dv) {
    const int64_t r1 = L / d1;
    if (r1 < 2) continue;
    consider({d1, r1});
    for (int64_t d2 : dv) {
      if (r1 % d2 != 0 || r1 / d2 < 2) continue;
      consider({d1, d2, r1 / d2});
    }
  }
  return !parts->empty();
}

// ---------------------------------------------------------------- tables
// Every table of a plan holds (cos a, sin a) of the angles a_m, m < count:
//   a_m = m * step                            (step != 0: the anchors of the omega refinement)
//   a_m = sign * 2 pi ((m * mult) mod P) / P  (otherwise; exact integer reduction first)
// stored as float2, double2, or float4 double-float pairs (cos hi, cos lo, sin hi, sin lo).
enum TableKind { TAB_F2 = 0, TAB_D2 = 1, TAB_DF4 = 2 };
struct TableSpec {
  int kind;
  int64_t count, mult, period;
  double step, sign;
};

static size_t table_elem_bytes(int kind) { return kind == TAB_F2 ? 8 : 16; }

__host__ __device__ inline double table_angle(const TableSpec& sp, int64_t m) {
  if (sp.step != 0.0) return (double)m * sp.step;
  const int64_t e = (m * sp.mult) % sp.period;
  return sp.sign * 2.0 * 3.14159265358979323846 * (double)e / (double)sp.period;
}

__host__ __device__ inline void table_store(const TableSpec& sp, void* out, int64_t m, double c, double s) {
  if (sp.kind == TAB_F2) {
    static_cast<float2*>(out)[m] = make_float2((float)c, (float)s);
  } else if (sp.kind == TAB_D2) {
    static_cast<double2*>(out)[m] = make_double2(c, s);
  } else {  // hi = RN(v), lo = RN(v - hi)
    const float ch = (float)c, sh = (float)s;
    static_cast<float4*>(out)[m] = make_float4(ch, (float)(c - (double)ch), sh, (float)(s - (double)sh));
  }
}

__global__ void table_kernel(TableSpec sp, void* out) {
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < sp.count;
       m += (int64_t)gridDim.x * blockDim.x) {
    const double a = table_angle(sp, m);
    table_store(sp, out, m, cos(a), sin(a));
  }
}

// One table into *dev.  dst == nullptr: computed on the host and copied into a cudaMalloc'd
// buffer (synchronous).  Otherwise carved from the caller's region (256-byte aligned) and
// generated on the device on dst->st (asynchronous, no allocation); with dst->base == nullptr
// only the bytes are counted.
static qw_status make_table(TableDst* dst, const TableSpec& sp, void** dev) {
  const size_t bytes = (size_t)sp.count * table_elem_bytes(sp.kind);
  if (!dst) {
    std::vector<unsigned char> h(bytes);
    for (int64_t m = 0; m < sp.count; ++m) {
      const double a = table_angle(sp, m);
      table_store(sp, h.data(), m, std::cos(a), std::sin(a));
    }
    QW_CHECK_CUDA(cudaMalloc(dev, bytes));
    QW_CHECK_CUDA(cudaMemcpy(*dev, h.data(), bytes, cudaMemcpyHostToDevice));
    return QW_OK;
  }
  const size_t off = (dst->used + 255) & ~size_t(255);
  dst->used = off + bytes;
  if (!dst->base) {
    *dev = nullptr;
    return QW_OK;
  }
  if (dst->used > dst->cap) {
    set_error("FFT tables need more than the %zu bytes given", dst->cap);
    return QW_ENOMEM;
  }
  *dev = dst->base + off;
  const int64_t blocks = std::min<int64_t>((sp.count + 255) / 256, 4096);
  table_kernel<<<(unsigned)std::max<int64_t>(1, blocks), 256, 0, dst->st>>>(sp, *dev);
  QW_CHECK_LAUNCH("table kernel launch");
  return QW_OK;
}

static TableSpec cis_spec(int kind, int64_t count, int64_t mult, int64_t period, double sign) {
  TableSpec sp;
  sp.kind = kind;
  sp.count = count;
  sp.mult = mult;
  sp.period = period;
  sp.step = 0.0;
  sp.sign = sign;
  return sp;
}

template <typename T>
static qw_status build_pass(FftPass* p, int L, int64_t S, int64_t O, int64_t tw_N, int64_t tw_div, bool twiddle,
                            TableDst* dst) {
  p->L = L;
  p->S = S;
  p->O = O;
  if (!radix_plan(L, p->radix, &p->nstages)) {
    set_error("FFT length %d is not 2^a 3^b", L);
    return QW_EINVAL;
  }
  const int esz = (int)sizeof(typename Cx<T>::t);
  // widest tile (<= 16 lines) whose two padded buffers fit the shared-memory budget
  const int64_t nlines = O * S;
  int C = 16;  // a power of two, so it divides the 256-thread block
  while (C > 1 && (C > nlines || 2 * (size_t)L * ((C % 2 == 0) ? C + 1 : C) * esz > (size_t)kFftSmemBytes)) C >>= 1;
  p->C = C;
  p->cshift = 0;
  while ((1 << p->cshift) < C) ++p->cshift;
  p->pitch = (C % 2 == 0) ? C + 1 : C;
  p->smem = 2 * (size_t)L * p->pitch * esz;
  if (p->smem > (size_t)kFftSmemBytes) {
    set_error("FFT line of %d elements does not fit shared memory", L);
    return QW_EINVAL;
  }
  p->twiddle = twiddle ? 1 : 0;
  p->tw_N = tw_N;
  p->tw_div = tw_div;
  p->tlo_bits = 12;
  // per-line table omega_L^m = exp(-2 pi i m / L), and the two-level table of omega_{tw_N}
  const int kind = sizeof(T) == 4 ? TAB_F2 : TAB_D2;
  qw_status st = make_table(dst, cis_spec(kind, L, 1, L, -1.0), &p->tw_line);
  if (st != QW_OK) return st;
  if (twiddle) {
    const int64_t T_lo = int64_t(1) << p->tlo_bits;
    st = make_table(dst, cis_spec(kind, T_lo, 1, tw_N, -1.0), &p->tw_lo);
    if (st != QW_OK) return st;
    st = make_table(dst, cis_spec(kind, (tw_N + T_lo - 1) / T_lo, T_lo, tw_N, -1.0), &p->tw_hi);
    if (st != QW_OK) return st;
  }
  return QW_OK;
}

template <typename T>
static qw_status fft_plan_t(FftPlan* f, const Geometry& g, TableDst* dst) {
  const int maxline = (sizeof(T) == 4) ? kMaxLineF32 : kMaxLineF64;
  f->npass = 0;
  const int P = g.ncoset * g.s;
  const int64_t ext[3] = {g.nx, g.ny, g.nz};
  for (int ax = 0; ax < g.dim && ax < 3; ++ax) {
    const int axis = (g.dim == 3) ? ax : ax;  // 3D: x, y, z; 2D: x, y; 1D: x
    const int64_t L = ext[axis];
    if (!fft_size_ok(L)) {
      set_error("spectral path needs 2^a 3^b axis lengths (got %lld)", (long long)L);
      return QW_EINVAL;
    }
    if (L == 1) {  // the DFT of length 1 is the identity: no pass
      FftAxis& A = f->axis[ax];
      A.nparts = 1;
      A.part[0] = 1;
      A.part[1] = A.part[2] = 1;
      A.first = f->npass;
      A.count = 0;
      continue;
    }
    std::vector<int> parts;
    if (!split_axis<T>(L, maxline, &parts)) {
      set_error("axis length %lld cannot be split into <= 3 passes of <= %d", (long long)L, maxline);
      return QW_EINVAL;
    }
    int64_t base = 1;  // stride of this axis
    for (int a = 0; a < axis; ++a) base *= ext[a];
    const int64_t outer_total = (int64_t)P * g.vol / (L * base);  // independent lines of this axis
    FftAxis& A = f->axis[ax];
    A.nparts = (int)parts.size();
    for (size_t q = 0; q < parts.size(); ++q) A.part[q] = parts[q];
    A.first = f->npass;
    // pass q transforms digit q: length parts[q], stride = base * prod(parts[q+1..]),
    // segments of length seg = parts[q] * stride repeat over outer * prod(parts[..q-1])
    int64_t seg = L * base;
    int64_t before = 1;
    for (size_t q = 0; q < parts.size(); ++q) {
      const int64_t Lq = parts[q];
      const int64_t stride = seg / Lq;
      const int64_t O = outer_total * before;
      const bool tw = (q + 1 < parts.size());
      qw_status st = build_pass<T>(&f->pass[f->npass], (int)Lq, stride, O, seg / base, base, tw, dst);
      if (st != QW_OK) return st;
      f->npass++;
      seg = stride;
      before *= Lq;
    }
    A.count = f->npass - A.first;
  }
  return QW_OK;
}

static qw_status trig_tables(FftPlan* f, const Geometry& g, TableDst* dst) {
  const int64_t ext[3] = {g.nx, g.ny, g.nz};
  qw_status st;
  for (int ax = 0; ax < g.dim; ++ax) {
    int64_t len, period;  // angle = 2 pi q / period for q < len
    if (g.dim == 1) {
      len = g.nx;
      period = g.nx;
    } else if (g.dim == 2) {
      if (ax > 0) break;  // one table serves both halves
      len = 2 * g.nx;
      period = 2 * g.nx;
    } else {
      len = ext[ax];
      period = 2 * ext[ax];
    }
    if ((st = make_table(dst, cis_spec(TAB_D2, len, 1, period, 1.0), &f->trig[ax])) != QW_OK) return st;
    if ((st = make_table(dst, cis_spec(TAB_F2, len, 1, period, 1.0), &f->trig32[ax])) != QW_OK) return st;
  }
  // anchors theta_j = j * kAngleStep, j <= kAngleTab (the same product the device forms)
  TableSpec anchors = cis_spec(TAB_D2, kAngleTab + 1, 1, 1, 1.0);
  anchors.step = kAngleStep;
  if ((st = make_table(dst, anchors, &f->angle)) != QW_OK) return st;
  // double-float tables: hi = RN(v), lo = RN(v - hi)
  if (g.dim == 1) {
    // the chain in two levels: angle 2 pi (kDfFine q1 + q0) / N
    const int64_t N = g.nx, B = kDfFine, nc = (N + B - 1) / B;
    if ((st = make_table(dst, cis_spec(TAB_DF4, B, 1, N, 1.0), &f->trigdf[0])) != QW_OK) return st;
    if ((st = make_table(dst, cis_spec(TAB_DF4, nc, B, N, 1.0), &f->trigdf[1])) != QW_OK) return st;
  } else {
    for (int ax = 0; ax < (g.dim == 2 ? 1 : 3); ++ax) {
      // the same angles as trig[ax]: 2D pi q / N (q < 2N), BCC pi q / M (q < M)
      const int64_t len = g.dim == 2 ? 2 * g.nx : ext[ax];
      const int64_t period = g.dim == 2 ? 2 * g.nx : 2 * ext[ax];
      if ((st = make_table(dst, cis_spec(TAB_DF4, len, 1, period, 1.0), &f->trigdf[ax])) != QW_OK) return st;
    }
  }
  anchors.kind = TAB_DF4;
  return make_table(dst, anchors, &f->angdf);
}

qw_status fft_plan_create(FftPlan* f, const Geometry& g, qw_dtype dt, TableDst* dst) {
  *f = FftPlan();
  f->dtype = dt;
  f->external_tables = dst != nullptr;
  f->field_bytes = (size_t)g.elems * (dt == QW_C64 ? 8 : 16);
  qw_status st = dt == QW_C64 ? fft_plan_t<float>(f, g, dst) : fft_plan_t<double>(f, g, dst);
  if (st != QW_OK) return st;
  return trig_tables(f, g, dst);
}

size_t fft_plan_table_bytes(const Geometry& g, qw_dtype dt) {
  TableDst count;  // base == nullptr: count only
  FftPlan f;
  if (fft_plan_create(&f, g, dt, &count) != QW_OK) return 0;
  return count.used;
}

void fft_plan_destroy(FftPlan* f) {
  if (f->external_tables) {  // the tables live in the caller's region
    *f = FftPlan();
    return;
  }
  for (int a = 0; a < 3; ++a) {
    if (f->trig[a]) cudaFree(f->trig[a]);
    if (f->trig32[a]) cudaFree(f->trig32[a]);
    f->trig[a] = nullptr;
    f->trig32[a] = nullptr;
  }
  if (f->angle) cudaFree(f->angle);
  f->angle = nullptr;
  for (int a = 0; a < 3; ++a) {
    if (f->trigdf[a]) cudaFree(f->trigdf[a]);
    f->trigdf[a] = nullptr;
  }
  if (f->angdf) cudaFree(f->angdf);
  f->angdf = nullptr;
  for (int i = 0; i < f->npass; ++i) {
    if (f->pass[i].tw_line) cudaFree(f->pass[i].tw_line);
    if (f->pass[i].tw_hi) cudaFree(f->pass[i].tw_hi);
    if (f->pass[i].tw_lo) cudaFree(f->pass[i].tw_lo);
  }
  f->npass = 0;
}

template <typename T, bool INV>
static qw_status run_pass(const FftPass& p, void* data, cudaStream_t st, const void* src = nullptr) {
  using V = typename Cx<T>::t;
  qw_status s2;
  if (run_2f<T, INV>(p.L, &p, data, src ? src : data, st, &s2)) return s2;
  if (src && src != data) {  // the Stockham kernel works in place: copy first
    const size_t bytes = (size_t)(p.O * p.S) * p.L * sizeof(V);
    QW_CHECK_CUDA(cudaMemcpyAsync(data, src, bytes, cudaMemcpyDeviceToDevice, st));
  }
  const qw_status sa = smem_attr(fft_pass_kernel<T, INV>, kFftSmemBytes + 64);
  if (sa != QW_OK) return sa;
  const int64_t nlines = p.O * p.S;
  const int64_t grid = (nlines + p.C - 1) / p.C;
  if (grid > 0x7fffffff) {
    set_error("FFT grid too large");
    return QW_EINVAL;
  }
  fft_pass_kernel<T, INV><<<(unsigned)grid, 256, p.smem, st>>>(static_cast<V*>(data), p,
                                                               static_cast<const V*>(p.tw_line),
                                                               static_cast<const V*>(p.tw_hi),
                                                               static_cast<const V*>(p.tw_lo));
  QW_CHECK_LAUNCH("fft pass launch");
  return QW_OK;
}

qw_status fft_forward_axis(const FftPlan& f, int ax, void* data, cudaStream_t st) {
  const FftAxis& A = f.axis[ax];
  for (int q = 0; q < A.count; ++q) {
    const FftPass& p = f.pass[A.first + q];
    qw_status s = f.dtype == QW_C64 ? run_pass<float, false>(p, data, st) : run_pass<double, false>(p, data, st);
    if (s != QW_OK) return s;
  }
  return QW_OK;
}

qw_status fft_forward_axis_from(const FftPlan& f, int ax, const void* src, void* dst, cudaStream_t st) {
  const FftAxis& A = f.axis[ax];
  if (A.count == 0 && src != dst)
    QW_CHECK_CUDA(cudaMemcpyAsync(dst, src, f.field_bytes, cudaMemcpyDeviceToDevice, st));
  for (int q = 0; q < A.count; ++q) {
    const FftPass& p = f.pass[A.first + q];
    const void* from = q == 0 ? src : nullptr;
    qw_status s = f.dtype == QW_C64 ? run_pass<float, false>(p, dst, st, from)
                                    : run_pass<double, false>(p, dst, st, from);
    if (s != QW_OK) return s;
  }
  return QW_OK;
}

qw_status fft_inverse_axis(const FftPlan& f, int ax, void* data, cudaStream_t st) {
  const FftAxis& A = f.axis[ax];
  for (int q = A.count - 1; q >= 0; --q) {
    const FftPass& p = f.pass[A.first + q];
    qw_status s = f.dtype == QW_C64 ? run_pass<float, true>(p, data, st) : run_pass<double, true>(p, data, st);
    if (s != QW_OK) return s;
  }
  return QW_OK;
}

qw_status fft_forward(const FftPlan& f, int dim, void* data, cudaStream_t st) {
  for (int ax = 0; ax < dim; ++ax) {
    qw_status s = fft_forward_axis(f, ax, data, st);
    if (s != QW_OK) return s;
  }
  return QW_OK;
}

qw_status fft_inverse(const FftPlan& f, int dim, void* data, cudaStream_t st) {
  for (int ax = dim - 1; ax >= 0; --ax) {
    qw_status s = fft_inverse_axis(f, ax, data, st);
    if (s != QW_OK) return s;
  }
  return QW_OK;
}

}  // namespace qw
