// Register DFT building blocks shared by the FFT passes (fft.cu) and the fused
// spectral kernel (spectral.cu): complex helpers, small DFTs, compile-time
// composite DFTs, and the two register steps of a line of length R1 * R2 held in
// shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qw {

// (L, R1, R2) of the register-kernel line lengths L = R1 * R2: powers of two (both
// precisions), then the lengths with a factor 3 (complex64 only).
#define QW_REG_LENGTHS_POW2(X) X(16, 4, 4) X(32, 8, 4) X(64, 8, 8) X(128, 16, 8) X(256, 16, 16)
#define QW_REG_LENGTHS_F32(X) \
  X(12, 4, 3) X(18, 6, 3) X(24, 8, 3) X(27, 9, 3) X(36, 6, 6) X(48, 8, 6) \
  X(54, 9, 6) X(72, 9, 8) X(81, 9, 9) X(96, 12, 8) X(108, 12, 9) X(144, 12, 12) \
  X(162, 18, 9) X(192, 16, 12) X(216, 18, 12) X(243, 27, 9) X(288, 18, 16) X(324, 18, 18) \
  X(384, 24, 16) X(432, 24, 18) X(512, 32, 16)

template <typename T> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };

template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
  V r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename V>
__device__ __forceinline__ V cmulc(V a, V b) {  // a * conj(b)
  V r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.y * b.x - a.x * b.y;
  return r;
}
template <typename V>
__device__ __forceinline__ V cadd(V a, V b) {
  a.x += b.x;
  a.y += b.y;
  return a;
}
template <typename V>
__device__ __forceinline__ V csub(V a, V b) {
  a.x -= b.x;
  a.y -= b.y;
  return a;
}
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename V>
__device__ __forceinline__ V mul_mi(V a) {
  V r;
  if (INV) {
    r.x = -a.y;
    r.y = a.x;
  } else {
    r.x = a.y;
    r.y = -a.x;
  }
  return r;
}

template <bool INV, typename V>
__device__ __forceinline__ void dft2(V& a0, V& a1) {
  V t = a0;
  a0 = cadd(t, a1);
  a1 = csub(t, a1);
}

template <bool INV, typename V>
__device__ __forceinline__ void dft4(V& a0, V& a1, V& a2, V& a3) {
  V s02 = cadd(a0, a2), d02 = csub(a0, a2);
  V s13 = cadd(a1, a3), d13 = mul_mi<INV>(csub(a1, a3));
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, d13);
  a3 = csub(d02, d13);
}

template <bool INV, typename T, typename V>
__device__ __forceinline__ void dft3(V& a0, V& a1, V& a2) {
  const T h = (T)0.86602540378443864676;  // sqrt(3)/2
  V t1 = cadd(a1, a2), t2 = csub(a1, a2);
  V b0 = cadd(a0, t1);
  V m;
  m.x = a0.x - (T)0.5 * t1.x;
  m.y = a0.y - (T)0.5 * t1.y;
  // forward: X1 = m - i h t2, X2 = m + i h t2 (inverse swaps)
  V r;
  r.x = h * t2.y;
  r.y = -h * t2.x;  // -i h t2
  if (INV) {
    r.x = -r.x;
    r.y = -r.y;
  }
  a0 = b0;
  a1 = cadd(m, r);
  a2 = csub(m, r);
}

template <bool INV, typename T, typename V>
__device__ __forceinline__ void dft8(V (&a)[8]) {
  // even/odd split into two radix-4 transforms
  dft4<INV>(a[0], a[2], a[4], a[6]);
  dft4<INV>(a[1], a[3], a[5], a[7]);
  const T r2 = (T)0.70710678118654752440;
  // twiddles w8^k, w8 = exp(-+ 2 pi i / 8)
  V o1 = a[3], o2 = a[5], o3 = a[7];
  V w1, w3;
  if (INV) {
    w1.x = r2 * (o1.x - o1.y);
    w1.y = r2 * (o1.x + o1.y);
    w3.x = -r2 * (o3.x + o3.y);
    w3.y = r2 * (o3.x - o3.y);
  } else {
    w1.x = r2 * (o1.x + o1.y);
    w1.y = r2 * (o1.y - o1.x);
    w3.x = r2 * (o3.y - o3.x);
    w3.y = -r2 * (o3.x + o3.y);
  }
  V w2 = mul_mi<INV>(o2);
  V e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6], o0 = a[1];
  a[0] = cadd(e0, o0);
  a[4] = csub(e0, o0);
  a[1] = cadd(e1, w1);
  a[5] = csub(e1, w1);
  a[2] = cadd(e2, w2);
  a[6] = csub(e2, w2);
  a[3] = cadd(e3, w3);
  a[7] = csub(e3, w3);
}

// omega_N^m = exp(-2 pi i m / N) from the two-level table (m < N)
template <typename V>
__device__ __forceinline__ V twiddle_big(const V* hi, const V* lo, int64_t m, int tlo_bits) {
  const int64_t mh = m >> tlo_bits;
  const int64_t ml = m & ((int64_t(1) << tlo_bits) - 1);
  return cmul(hi[mh], lo[ml]);
}

// ------------------------------------------------- two-factor register kernel
// Lines of length L = R1 * R2 (R1, R2 in 4, 8, 16): n = n1 + R1 n2,
//   Y[n1][k2] = omega_L^{n1 k2} sum_{n2} x[n1 + R1 n2] omega_{R2}^{n2 k2}   (step A, registers)
//   X[k2 + R2 k1] = sum_{n1} Y[n1][k2] omega_{R1}^{n1 k1}                   (step B, registers)
// with one shared-memory exchange between the steps; index maps are
// compile-time, so the per-element cost is the butterflies, not the indexing.
template <int R, bool INV, typename T, typename V> struct RegDFT;
template <bool INV, typename T, typename V> struct RegDFT<2, INV, T, V> {
  __device__ __forceinline__ static void run(V (&a)[2]) { dft2<INV>(a[0], a[1]); }
};
template <bool INV, typename T, typename V> struct RegDFT<4, INV, T, V> {
  __device__ __forceinline__ static void run(V (&a)[4]) { dft4<INV>(a[0], a[1], a[2], a[3]); }
};
template <bool INV, typename T, typename V> struct RegDFT<8, INV, T, V> {
  __device__ __forceinline__ static void run(V (&a)[8]) { dft8<INV, T>(a); }
};
template <bool INV, typename T, typename V> struct RegDFT<16, INV, T, V> {
  __device__ __forceinline__ static void run(V (&a)[16]) {
    // even / odd halves, then X_k = E_k + w16^k O_k, X_{k+8} = E_k - w16^k O_k
    V e[8], o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      e[j] = a[2 * j];
      o[j] = a[2 * j + 1];
    }
    dft8<INV, T>(e);
    dft8<INV, T>(o);
    const T cs[8] = {(T)1.0, (T)0.92387953251128675613, (T)0.70710678118654752440, (T)0.38268343236508977173,
                     (T)0.0, (T)-0.38268343236508977173, (T)-0.70710678118654752440, (T)-0.92387953251128675613};
    const T sn[8] = {(T)0.0, (T)0.38268343236508977173, (T)0.70710678118654752440, (T)0.92387953251128675613,
                     (T)1.0, (T)0.92387953251128675613, (T)0.70710678118654752440, (T)0.38268343236508977173};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      V w;  // w16^k = cos - i sin (forward), cos + i sin (inverse)
      w.x = cs[k];
      w.y = INV ? sn[k] : -sn[k];
      const V t = (k == 0) ? o[0] : cmul(o[k], w);
      a[k] = cadd(e[k], t);
      a[k + 8] = csub(e[k], t);
    }
  }
};

// Compile-time twiddles exp(-2 pi i m / R) for the composite register DFTs:
// cos and sin of 2 pi m / R by a Taylor series after reduction to [-pi/4, pi/4]
// (double precision; the values become immediates).
constexpr double ce_pi = 3.14159265358979323846264338327950288;
constexpr double ce_taylor_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 14; ++k) {
    term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
constexpr double ce_taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 14; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}
// angle 2 pi m / R, m in [0, R): octant reduction with exact rational arithmetic
constexpr double ce_trig(int m, int R, bool want_sin) {
  const int num = 8 * m, q = num / R;                  // octant
  const double f = (double)(num - q * R) / (double)R;  // fraction of an octant
  const double x = f * ce_pi / 4.0;
  const double sx = ce_taylor_sin(x), cx = ce_taylor_cos(x);
  const double sy = ce_taylor_sin(ce_pi / 4.0 - x), cy = ce_taylor_cos(ce_pi / 4.0 - x);
  double s = 0.0, c = 0.0;
  switch (q & 7) {
    case 0: s = sx; c = cx; break;
    case 1: s = cy; c = sy; break;
    case 2: s = cx; c = -sx; break;
    case 3: s = sy; c = -cy; break;
    case 4: s = -sx; c = -cx; break;
    case 5: s = -cy; c = -sy; break;
    case 6: s = -cx; c = sx; break;
    default: s = -sy; c = cy; break;
  }
  return want_sin ? s : c;
}

constexpr int reg_first_factor(int R) {
  // split R = P * Q with Q the factor transformed first
  return (R % 16 == 0 && R > 16) ? 16 : (R % 8 == 0 && R > 8) ? 8 : (R % 4 == 0 && R > 4) ? 4
       : (R % 3 == 0 && R > 3) ? R / 3 : (R % 2 == 0 && R > 2) ? 2 : R;
}

template <bool INV, typename T, typename V> struct RegDFT<3, INV, T, V> {
  __device__ __forceinline__ static void run(V (&a)[3]) { dft3<INV, T>(a[0], a[1], a[2]); }
};

// Composite R = P * Q (P = reg_first_factor(R)): Q-point DFTs over a[p + P q],
// twiddle exp(-+2 pi i p k2 / R), P-point DFTs over p; output index k2 + Q k1.
// The (p, k2) loops are template recursions so every twiddle is a constant.
template <int R, int Q, int p, int k2, bool INV, typename T, typename V>
struct TwApply {
  __device__ __forceinline__ static void run(const V (&b)[Q], V (&t)[R]) {
    if constexpr (k2 < Q) {
      constexpr int m = (p * k2) % R;
      if constexpr (m == 0) {
        t[p * Q + k2] = b[k2];
      } else {
        constexpr double c = ce_trig(m, R, false), sn = ce_trig(m, R, true);
        V w;
        w.x = (T)c;
        w.y = INV ? (T)sn : (T)-sn;
        t[p * Q + k2] = cmul(b[k2], w);
      }
      TwApply<R, Q, p, k2 + 1, INV, T, V>::run(b, t);
    }
  }
};

template <int R, int P, int Q, int p, bool INV, typename T, typename V>
struct StepA {
  __device__ __forceinline__ static void run(const V (&a)[R], V (&t)[R]) {
    if constexpr (p < P) {
      V b[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) b[q] = a[p + P * q];
      RegDFT<Q, INV, T, V>::run(b);
      TwApply<R, Q, p, 0, INV, T, V>::run(b, t);
      StepA<R, P, Q, p + 1, INV, T, V>::run(a, t);
    }
  }
};

template <int R, bool INV, typename T, typename V>
struct RegDFT {
  static constexpr int P = reg_first_factor(R);
  static constexpr int Q = R / P;
  __device__ __forceinline__ static void run(V (&a)[R]) {
    V t[R];
    StepA<R, P, Q, 0, INV, T, V>::run(a, t);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) {
      V c[P];
#pragma unroll
      for (int p = 0; p < P; ++p) c[p] = t[p * Q + k2];
      RegDFT<P, INV, T, V>::run(c);
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) a[k2 + Q * k1] = c[k1];
    }
  }
};

// Global -> shared copy of one complex element without a register round trip
// (cp.async; a source size of 0 writes zeros), and the wait for this thread's copies.
template <typename V>
__device__ __forceinline__ void cp_async_elem(V* dst, const V* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const unsigned n = valid ? (unsigned)sizeof(V) : 0u;
  if constexpr (sizeof(V) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Step-A twiddles read from the table omega_L^m (m < L) when needed, instead of
// being held in registers.
template <typename V>
struct TwRow {
  const V* __restrict__ tab;
  int r;
  __device__ __forceinline__ V operator[](int k2) const { return tab[r * k2]; }
};

// The two register steps of the length R1 * R2 transform of line c, element n at
// sm[c + CP n] (natural order in, natural order out); thread r of the line works
// in both steps (r < R1 in step A, r < R2 in step B).  tw[k2] = omega_L^{r k2}
// (k2 >= 1) are the step-A twiddles of this thread: a register array, or a
// TwRow reading them from the per-line table.  The caller synchronises the
// CTA before; the steps end with a CTA-wide barrier.
template <typename T, bool INV, int R1, int R2, int CP, typename TW>
__device__ __forceinline__ void reg_fft_steps(typename Cx<T>::t* sm, int c, int r, const TW& tw) {
  using V = typename Cx<T>::t;
  // ---- step A: thread r = n1 < R1
  V a[R2];
  if (r < R1) {
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) a[n2] = sm[c + CP * (r + R1 * n2)];
    RegDFT<R2, INV, T, V>::run(a);
#pragma unroll
    for (int k2 = 1; k2 < R2; ++k2) a[k2] = INV ? cmulc(a[k2], tw[k2]) : cmul(a[k2], tw[k2]);
  }
  __syncthreads();
  if (r < R1) {
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) sm[c + CP * (r * R2 + k2)] = a[k2];
  }
  __syncthreads();
  // ---- step B: thread r = k2 < R2
  V b[R1];
  if (r < R2) {
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) b[n1] = sm[c + CP * (n1 * R2 + r)];
    RegDFT<R1, INV, T, V>::run(b);
  }
  __syncthreads();
  if (r < R2) {
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) sm[c + CP * (r + R2 * k1)] = b[k1];
  }
  __syncthreads();
}

}  // namespace qw
