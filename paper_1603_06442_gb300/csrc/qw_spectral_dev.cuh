// Device side of the Fourier form shared by spectral.cu and the fused-x-pass
// instantiation units (fused_x_*.cu): symbols, D_k^t per wave vector, particle-weight
// sums, double-float omega_k, and the fused x pass kernel with its launcher template
// (instantiated per line length in the fused_x_*.cu files so they compile in parallel).
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "qw_internal.cuh"
#include "qw_regdft.cuh"

namespace qw {


template <typename T> struct Cx2;
template <> struct Cx2<float> { using t = float2; };
template <> struct Cx2<double> { using t = double2; };

template <typename V, typename T>
__device__ __forceinline__ V make_vec(V v, T s) {
  v.x *= s;
  v.y *= s;
  return v;
}

struct AxesDev {
  int nparts[3];
  int part[3][3];
  int64_t len[3];
  const double2* trig[3];
  const float2* trig32[3];
  const double2* angle;
  const float4* trigdf[3];
  const float4* angdf;
};

inline AxesDev to_dev(const SpecAxes& a) {
  AxesDev d;
  for (int ax = 0; ax < 3; ++ax) {
    d.nparts[ax] = a.nparts[ax];
    d.len[ax] = a.len[ax];
    for (int q = 0; q < 3; ++q) d.part[ax][q] = a.part[ax][q];
    d.trig[ax] = a.trig[ax];
    d.trig32[ax] = a.trig32[ax];
  }
  d.angle = a.angle;
  for (int ax = 0; ax < 3; ++ax) d.trigdf[ax] = a.trigdf[ax];
  d.angdf = a.angdf;
  return d;
}

// Mass coefficients n = sqrt(1 - m^2) and m in both precisions, and the step count t
// (with its FP32 copy when t < 2^24), so that complex64 kernels convert nothing on
// the FP64 pipe (FP64 runs at ~1/64 of the FP32 rate on this part).
struct Mass {
  double n, m;
  float nf, mf;
  float2 n_df, n2_df, m2_df;  // n, n^2, m^2 as double-float (hi, lo)
};
struct TimeArg {
  double tt;
  float tf;
  int small;  // t < 2^24: the split-nu phase applies
  int odd;    // t odd: (-1)^t = -1
};
inline float2 split_df(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}
inline Mass make_mass(double n, double m) {
  return Mass{n, m, (float)n, (float)m, split_df(n), split_df(n * n), split_df(m * m)};
}
inline TimeArg make_time(int64_t t) {
  return TimeArg{(double)t, (float)t, t < (int64_t(1) << 24) ? 1 : 0, (int)(t & 1)};
}

// Frequency index of storage position p on an axis split into digits
// (A), (A, B) or (A, B1, B2): the passes leave frequency k1 + A k2 at B k1 + k2
// (and, recursively, k1 + A (k1' + B1 k2') at B k1 + B2 k1' + k2').
__device__ __forceinline__ int64_t freq_of(int64_t p, const AxesDev& a, int ax) {
  const int np = a.nparts[ax];
  if (np == 1) return p;
  const int64_t A = a.part[ax][0];
  const int64_t B = a.len[ax] / A;
  const int64_t k1 = p / B, r = p - k1 * B;
  if (np == 2) return k1 + A * r;
  const int64_t B1 = a.part[ax][1], B2 = a.part[ax][2];
  const int64_t k1b = r / B2, k2b = r - k1b * B2;
  return k1 + A * (k1b + B1 * k2b);
}

// ---------------------------------------------------------------- symbols
// u_k, n~_k from the per-axis (cos, sin) tables: the frequency indices select
// exact table angles (q = 1 adds pi to the x half-angle: the BCC wave vector q1).
template <typename T>
__device__ __forceinline__ void tab(const AxesDev& a, int ax, int64_t i, T& c, T& s) {
  if (sizeof(T) == 8) {
    const double2 e = a.trig[ax][i];
    c = (T)e.x;
    s = (T)e.y;
  } else {
    const float2 e = a.trig32[ax][i];
    c = (T)e.x;
    s = (T)e.y;
  }
}

template <typename T>
__device__ __forceinline__ void symbol_tab(int dim, const AxesDev& a, int64_t fx, int64_t fy, int64_t fz, int q,
                                           T& u, T& nx, T& ny, T& nz) {
  if (dim == 1) {
    T ec, es;
    tab<T>(a, 0, fx, ec, es);
    u = ec;
    nx = (T)0;
    ny = (T)0;
    nz = es;
  } else if (dim == 2) {
    const int64_t N2 = 2 * a.len[0];
    int64_t dm = fx - fy;
    if (dm < 0) dm += N2;
    T cx, sx, cy, sy;
    tab<T>(a, 0, fx + fy, cx, sx);
    tab<T>(a, 0, dm, cy, sy);
    u = cx * cy;
    nx = sx * cy;
    ny = cx * sy;
    nz = sx * sy;
  } else {
    T cx, sx, cy, sy, cz, sz;
    tab<T>(a, 0, fx, cx, sx);
    tab<T>(a, 1, fy, cy, sy);
    tab<T>(a, 2, fz, cz, sz);
    if (q) {
      cx = -cx;
      sx = -sx;
    }
    u = cx * cy * cz + sx * sy * sz;
    nx = sx * cy * cz - cx * sy * sz;
    ny = cx * sy * cz + sx * cy * sz;
    nz = cx * cy * sz - sx * sy * cz;
  }
}

// Wave vector(s) of storage position (x, y, z): k_j = 2 pi f_j / len_j with f the
// frequency index of the position; fsum = fx + fy + fz (BCC coset phase).
__device__ __forceinline__ void wave_vectors(int dim, int64_t x, int64_t y, int64_t z, const AxesDev& a,
                                             int64_t (&f)[3], int64_t& fsum) {
  f[0] = freq_of(x, a, 0);
  f[1] = dim >= 2 ? freq_of(y, a, 1) : 0;
  f[2] = dim >= 3 ? freq_of(z, a, 2) : 0;
  fsum = f[0] + f[1] + f[2];
}

// a = exp(i (k1 + k2 + k3)/2) = exp(i pi fx / M) exp(i pi fy / M) exp(i pi fz / M): the
// product of the three per-axis table entries (the half angles of the BCC symbol tables).
template <typename T>
__device__ __forceinline__ void coset_phase_tab(const AxesDev& a, const int64_t (&f)[3], T& ar, T& ai) {
  T c0, s0, c1, s1, c2, s2;
  tab<T>(a, 0, f[0], c0, s0);
  tab<T>(a, 1, f[1], c1, s1);
  tab<T>(a, 2, f[2], c2, s2);
  const T pr = c0 * c1 - s0 * s1, pi = c0 * s1 + s0 * c1;
  ar = pr * c2 - pi * s2;
  ai = pr * s2 + pi * c2;
}

template <typename T>
__device__ __forceinline__ void coset_phase(int64_t fsum, int64_t M, T& ar, T& ai) {
  const int64_t q = fsum % (2 * M);
  if (sizeof(T) == 8) {
    double s, c;
    sincospi((double)q / (double)M, &s, &c);
    ar = (T)c;
    ai = (T)s;
  } else {
    float s, c;
    sincospif((float)(int)q / (float)(int)M, &s, &c);  // 32-bit conversions (q < 2M <= 2^13)
    ar = (T)c;
    ai = (T)s;
  }
}

// Position of the thread in a 3D launch over (nx, ny, nz); false when outside.
__device__ __forceinline__ bool grid_pos(const AxesDev& a, int64_t& x, int64_t& y, int64_t& z) {
  x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  y = blockIdx.y;
  z = blockIdx.z;
  return x < a.len[0];
}

// (cos, sin)(2 pi nu t) for nu = hi + lo (FP32 pair) and integer t < 2^24, in FP32:
// p + e = hi t exactly (FMA), p - rint(p) is exact, lo t is below 2^-24 |p|.
__device__ __forceinline__ void phase_split(float2 nu, float tf, float& c, float& s) {
  const float p = nu.x * tf;
  const float e = fmaf(nu.x, tf, -p);
  const float r = (p - rintf(p)) + fmaf(nu.y, tf, e);
  sincospif(2.0f * r, &s, &c);
}

// (cos, sin) of omega t with omega t reduced modulo 2 pi in FP64.
__device__ __forceinline__ void phase(double omega, double tt, double& c, double& s) {
  const double TWO_PI_HI = 6.283185307179586232e+00;
  const double TWO_PI_LO = 2.449293598294706e-16;
  const double p = omega * tt;
  const double e = fma(omega, tt, -p);  // exact low part of the product
  const double kq = rint(p * 0.15915494309189533577);
  double r = fma(-kq, TWO_PI_HI, p);
  r = fma(-kq, TWO_PI_LO, r) + e;
  sincos(r, &s, &c);
}
// (cos, sin) of omega t for omega = hi + lo (double-double): hi t is split exactly into
// p + e (FMA), the low part adds lo t, and the reduction modulo 2 pi is that of phase();
// the reduced phase then carries ~1e-16 of rounding whatever t (t < 2^53), instead of
// t ulp(omega).
__device__ __forceinline__ void phase_dd(double hi, double lo, double tt, double& c, double& s) {
  const double TWO_PI_HI = 6.283185307179586232e+00;
  const double TWO_PI_LO = 2.449293598294706e-16;
  const double p = hi * tt;
  const double e = fma(hi, tt, -p);
  const double kq = rint(p * 0.15915494309189533577);
  double r = fma(-kq, TWO_PI_HI, p);
  r = fma(-kq, TWO_PI_LO, r) + (e + lo * tt);
  sincos(r, &s, &c);
}
// complex64 path: same FP64 reduction without the product's low part (about
// 1e-16 * omega t, far below the FP32 resolution of the reduced phase)
__device__ __forceinline__ void phase32(double omega, double tt, float& c, float& s) {
  const double TWO_PI_HI = 6.283185307179586232e+00;
  const double TWO_PI_LO = 2.449293598294706e-16;
  const double p = omega * tt;
  const double kq = rint(p * 0.15915494309189533577);
  double r = fma(-kq, TWO_PI_HI, p);
  r = fma(-kq, TWO_PI_LO, r);
  sincosf((float)r, &s, &c);
}

// w = G^ v for one wave vector, s = 2 or 4 components: (gx, gy, gz) = n n~ / sin(omega),
// gm = m / sin(omega).
template <typename T, int S>
__device__ __forceinline__ void ghat_mul(const typename Cx2<T>::t (&v)[S], T gx, T gy, T gz, T gm,
                                         typename Cx2<T>::t (&w)[S]) {
  using V = typename Cx2<T>::t;
  if (S == 2) {
    // G^ = [[gz, -gm], [-gm, -gz]] (1D: gz = n sin k / sin omega)
    w[0].x = gz * v[0].x - gm * v[1].x;
    w[0].y = gz * v[0].y - gm * v[1].y;
    w[1].x = -gm * v[0].x - gz * v[1].x;
    w[1].y = -gm * v[0].y - gz * v[1].y;
  } else {
    // sigma.n v for the upper (0,1) and lower (2,3) pairs
    V su0, su1, sl0, sl1;
    su0.x = gz * v[0].x + gx * v[1].x + gy * v[1].y;
    su0.y = gz * v[0].y + gx * v[1].y - gy * v[1].x;
    su1.x = gx * v[0].x - gy * v[0].y - gz * v[1].x;
    su1.y = gx * v[0].y + gy * v[0].x - gz * v[1].y;
    sl0.x = gz * v[2].x + gx * v[3].x + gy * v[3].y;
    sl0.y = gz * v[2].y + gx * v[3].y - gy * v[3].x;
    sl1.x = gx * v[2].x - gy * v[2].y - gz * v[3].x;
    sl1.y = gx * v[2].y + gy * v[2].x - gz * v[3].y;
    w[0].x = su0.x - gm * v[2].x;
    w[0].y = su0.y - gm * v[2].y;
    w[1].x = su1.x - gm * v[3].x;
    w[1].y = su1.y - gm * v[3].y;
    w[2].x = -gm * v[0].x - sl0.x;
    w[2].y = -gm * v[0].y - sl0.y;
    w[3].x = -gm * v[1].x - sl1.x;
    w[3].y = -gm * v[1].y - sl1.y;
  }
}

// out = cos(phi) v - i sin(phi) G^ v for one wave vector, s = 2 or 4 components.
template <typename T, int S>
__device__ __forceinline__ void apply_dt(typename Cx2<T>::t (&v)[S], T c, T s, T gn, T gx, T gy, T gz, T gm) {
  using V = typename Cx2<T>::t;
  V w[S];
  ghat_mul<T, S>(v, gx, gy, gz, gm, w);
  (void)gn;
#pragma unroll
  for (int q = 0; q < S; ++q) {
    // cos v - i sin w
    V r;
    r.x = c * v[q].x + s * w[q].y;
    r.y = c * v[q].y - s * w[q].x;
    v[q] = r;
  }
}

// G^ entries for one wave vector in precision T.
template <typename T>
__device__ __forceinline__ void ghat(int dim, const AxesDev& a, const int64_t (&f)[3], int q, const Mass& ms,
                                     T& gx, T& gy, T& gz, T& gm) {
  T u, nx, ny, nz;
  symbol_tab<T>(dim, a, f[0], f[1], f[2], q, u, nx, ny, nz);
  const T nf = sizeof(T) == 8 ? (T)ms.n : (T)ms.nf, mf = sizeof(T) == 8 ? (T)ms.m : (T)ms.mf;
  const T sw = sqrt(mf * mf + nf * nf * (nx * nx + ny * ny + nz * nz));
  const T inv = sw > (T)0 ? (T)1 / sw : (T)0;
  gx = nf * nx * inv;
  gy = nf * ny * inv;
  gz = nf * nz * inv;
  gm = mf * inv;
}

// omega = atan2(S, C) for S = sqrt(S2) >= 0, S^2 + C^2 = 1, to FP64 accuracy with
// few FP64 operations (FP64 runs at ~1/64 of the FP32 rate here):
//   S   : FP32 square root, one Newton correction in FP64;
//   w0  : FP32 atan2, only to pick the anchor theta_j = j pi / kAngleTab nearest omega;
//   x   = sin(omega - theta_j) = S cos theta_j - C sin theta_j (FP64, anchors from an FP64 table),
//         |x| <= pi / (2 kAngleTab) + 1e-6 < 1.6e-3;
//   omega = theta_j + asin(x),  asin(x) = x + x^3/6 + 3 x^5/40 + O(x^7)  (x^7 term < 1e-21).
__device__ __forceinline__ double omega_fast(double C, double S2, const double2* __restrict__ angle) {
  double S;
  if (S2 > 1e-30) {
    const float s0 = sqrtf((float)S2);
    const double e = fma(-(double)s0, (double)s0, S2);
    S = fma(e, (double)(0.5f / s0), (double)s0);
  } else {
    S = sqrt(S2);
  }
  const float w0 = atan2f((float)S, (float)C);
  int j = __float2int_rn(w0 * (float)(kAngleTab / 3.14159265358979323846));
  j = j < 0 ? 0 : (j > kAngleTab ? kAngleTab : j);
  const double2 an = angle[j];
  const double x = fma(S, an.x, -C * an.y);
  const double x2 = x * x;
  const double d = fma(x * x2, fma(x2, 0.075, 1.0 / 6.0), x);
  return (double)j * kAngleStep + d;
}

// omega_k in FP64 from the FP64 tables, computed in the kernel (served path: no table)
__device__ __forceinline__ double omega_of(int dim, const AxesDev& a, const int64_t (&f)[3], int q,
                                          const Mass& ms) {
  const double n = ms.n, m = ms.m;
  double u, nx, ny, nz;
  symbol_tab<double>(dim, a, f[0], f[1], f[2], q, u, nx, ny, nz);
  return omega_fast(n * u, m * m + n * n * (nx * nx + ny * ny + nz * nz), a.angle);
}

template <typename T, int S>
__device__ __forceinline__ void cs_of(double omega, double tt, T& c, T& s) {
  if (sizeof(T) == 8) {
    double cd, sd;
    phase(omega, tt, cd, sd);
    c = (T)cd;
    s = (T)sd;
  } else {
    float cf, sf;
    phase32(omega, tt, cf, sf);
    c = (T)cf;
    s = (T)sf;
  }
}

// ---------------------------------------------------------------- double-float
// Unevaluated pairs hi + lo of FP32 numbers (|lo| <= ulp(hi)/2, ~46-bit significand),
// built from error-free transformations (Knuth two-sum, FMA two-product); the _rn
// intrinsics keep the compiler from contracting or reordering them.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_fast_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return df_fast_sum(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_sum(p, e);
}
__device__ __forceinline__ DF df_of(float2 v) { return DF{v.x, v.y}; }

// (cos, sin) of a symbol-table angle in double-float (the tables of trig[]; the chain
// combines its two levels by the angle-addition formula)
__device__ __forceinline__ void tab_df(const AxesDev& a, int dim, int ax, int64_t i, DF& c, DF& s) {
  if (dim == 1) {
    const float4 f = a.trigdf[0][i & (kDfFine - 1)], g = a.trigdf[1][i / kDfFine];
    const DF c0{f.x, f.y}, s0{f.z, f.w}, c1{g.x, g.y}, s1{g.z, g.w};
    c = df_sub(df_mul(c1, c0), df_mul(s1, s0));
    s = df_add(df_mul(s1, c0), df_mul(c1, s0));
  } else {
    const float4 f = a.trigdf[ax][i];
    c = DF{f.x, f.y};
    s = DF{f.z, f.w};
  }
}

// nu_k = omega_k / (2 pi) in double-float without FP64 operations: the symbol
// (u, n~) and C = n u, S^2 = m^2 + n^2 |n~|^2 in double-float, S by an FP32 square root
// and one Newton correction, and omega = theta_j + asin(S cos theta_j - C sin theta_j)
// around the nearest anchor theta_j = j pi / kAngleTab (as omega_fast), so that
// nu = j / (2 kAngleTab) + asin(x) / (2 pi).  Error ~1e-13 in nu.
__device__ __forceinline__ float2 nu_df(int dim, const AxesDev& a, const int64_t (&f)[3], int q, const Mass& ms) {
  DF u, nx, ny, nz;
  if (dim == 1) {
    DF c, s;
    tab_df(a, 1, 0, f[0], c, s);
    u = c;
    nx = DF{0.f, 0.f};
    ny = nx;
    nz = s;
  } else if (dim == 2) {
    const int64_t N2 = 2 * a.len[0];
    int64_t dm = f[0] - f[1];
    if (dm < 0) dm += N2;
    DF cx, sx, cy, sy;
    tab_df(a, 2, 0, f[0] + f[1], cx, sx);
    tab_df(a, 2, 0, dm, cy, sy);
    u = df_mul(cx, cy);
    nx = df_mul(sx, cy);
    ny = df_mul(cx, sy);
    nz = df_mul(sx, sy);
  } else {
    DF cx, sx, cy, sy, cz, sz;
    tab_df(a, 3, 0, f[0], cx, sx);
    tab_df(a, 3, 1, f[1], cy, sy);
    tab_df(a, 3, 2, f[2], cz, sz);
    if (q) {
      cx = df_neg(cx);
      sx = df_neg(sx);
    }
    const DF cxcy = df_mul(cx, cy), sxsy = df_mul(sx, sy), cxsy = df_mul(cx, sy), sxcy = df_mul(sx, cy);
    u = df_add(df_mul(cxcy, cz), df_mul(sxsy, sz));
    nx = df_sub(df_mul(sxcy, cz), df_mul(cxsy, sz));
    ny = df_add(df_mul(cxsy, cz), df_mul(sxcy, sz));
    nz = df_sub(df_mul(cxcy, sz), df_mul(sxsy, cz));
  }
  const DF C = df_mul(df_of(ms.n_df), u);
  const DF nn = df_add(df_add(df_mul(nx, nx), df_mul(ny, ny)), df_mul(nz, nz));
  const DF S2 = df_add(df_of(ms.m2_df), df_mul(df_of(ms.n2_df), nn));
  DF S{0.f, 0.f};
  if (S2.hi > 0.f) {
    const float s0 = sqrtf(S2.hi);
    const float p = __fmul_rn(s0, s0), e = __fmaf_rn(s0, s0, -p);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(S2.hi, p), e), S2.lo);  // S2 - s0^2
    S = df_fast_sum(s0, __fmul_rn(r, __fdiv_rn(0.5f, s0)));
  }
  const float w0 = atan2f(S.hi, C.hi);
  int j = __float2int_rn(w0 * (float)(kAngleTab / 3.14159265358979323846));
  j = j < 0 ? 0 : (j > kAngleTab ? kAngleTab : j);
  const float4 an = a.angdf[j];
  const DF x = df_sub(df_mul(S, DF{an.x, an.y}), df_mul(C, DF{an.z, an.w}));  // sin(omega - theta_j)
  const float xf = x.hi, x2 = xf * xf;
  const float cub = xf * x2 * fmaf(x2, 0.075f, 1.0f / 6.0f);  // asin(x) - x, < 7e-10
  const DF d = df_add(x, DF{cub, 0.f});
  const DF inv2pi{1.591549367e-01f, 6.420638243e-09f};          // 1 / (2 pi) in double-float
  const DF nu = df_add(DF{(float)j * (0.5f / kAngleTab), 0.f}, df_mul(d, inv2pi));
  return make_float2(nu.hi, nu.lo);
}

// cos, sin of omega_k t for wave vector q of storage index idx: from the plan's table
// (FP64 omega; for complex64 the split nu table, t < 2^24) or computed here (no table).
template <typename T, int S>
__device__ __forceinline__ void cs_at(int dim, const AxesDev& a, const int64_t (&f)[3], int q, int64_t slot,
                                      const Mass& ms, const double* __restrict__ omega, const TimeArg& ta, T& c,
                                      T& s) {
  if (omega == nullptr) {
    if (sizeof(T) == 4 && ta.small) {
      float cf, sf;
      phase_split(nu_df(dim, a, f, q, ms), ta.tf, cf, sf);
      c = (T)cf;
      s = (T)sf;
    } else {
      cs_of<T, S>(omega_of(dim, a, f, q, ms), ta.tt, c, s);
    }
  } else if (sizeof(T) == 8) {
    // complex128 plans store omega_k as a double-double (hi, lo)
    const double2 w = reinterpret_cast<const double2*>(omega)[slot];
    double cd, sd;
    phase_dd(w.x, w.y, ta.tt, cd, sd);
    c = (T)cd;
    s = (T)sd;
  } else {
    const float2 nu = reinterpret_cast<const float2*>(omega)[slot];
    if (ta.small) {
      float cf, sf;
      phase_split(nu, ta.tf, cf, sf);
      c = (T)cf;
      s = (T)sf;
    } else {
      cs_of<T, S>(6.283185307179586232 * ((double)nu.x + (double)nu.y), ta.tt, c, s);
    }
  }
}

// D_k^t, times the scale (1/|V|, optionally the initial norm), on the spectral values
// of storage position (x, y, z) (storage index idx): v[0..s) in 1D/2D, and in BCC the
// two cosets' four components v[0..4) (coset 0) and v[4..8) (coset 1).
template <typename T>
__device__ __forceinline__ void evolve_point(int dim, const AxesDev& a, int64_t x, int64_t y, int64_t z,
                                             int64_t idx, const Mass& ms, const double* __restrict__ omega,
                                             const TimeArg& ta, T scale, typename Cx2<T>::t (&v)[8]) {
  using V = typename Cx2<T>::t;
  int64_t f[3], fs;
  wave_vectors(dim, x, y, z, a, f, fs);
  if (dim == 1) {
    V w[2] = {v[0], v[1]};
    T c, s, gx, gy, gz, gm;
    cs_at<T, 2>(1, a, f, 0, idx, ms, omega, ta, c, s);
    ghat<T>(1, a, f, 0, ms, gx, gy, gz, gm);
    apply_dt<T, 2>(w, c, s, (T)0, gx, gy, gz, gm);
    v[0] = make_vec(w[0], scale);
    v[1] = make_vec(w[1], scale);
  } else if (dim == 2) {
    V w[4] = {v[0], v[1], v[2], v[3]};
    T c, s, gx, gy, gz, gm;
    cs_at<T, 4>(2, a, f, 0, idx, ms, omega, ta, c, s);
    ghat<T>(2, a, f, 0, ms, gx, gy, gz, gm);
    apply_dt<T, 4>(w, c, s, (T)0, gx, gy, gz, gm);
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = make_vec(w[q], scale);
  } else {
    T ar, ai;
    coset_phase_tab<T>(a, f, ar, ai);  // a = exp(i (k1 + k2 + k3)/2)
    V c0[4], c1[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      // a* Psi1
      V b;
      b.x = ar * v[4 + q].x + ai * v[4 + q].y;
      b.y = ar * v[4 + q].y - ai * v[4 + q].x;
      c0[q].x = (T)0.5 * (v[q].x + b.x);
      c0[q].y = (T)0.5 * (v[q].y + b.y);
      c1[q].x = (T)0.5 * (v[q].x - b.x);
      c1[q].y = (T)0.5 * (v[q].y - b.y);
    }
    {
      // q1 = q0 + (pi, 0, 0) flips the signs of u and n~ (the x half angle moves by pi), so
      // omega_q1 = pi - omega_q0 and D_q1 = -Gamma D_q0 Gamma with Gamma = diag(I, -I):
      // D_q1^t = (-1)^t Gamma D_q0^t Gamma.  One phase and one G^ serve both half spectra.
      T c, s, gx, gy, gz, gm;
      cs_at<T, 4>(3, a, f, 0, idx, ms, omega, ta, c, s);
      ghat<T>(3, a, f, 0, ms, gx, gy, gz, gm);
      apply_dt<T, 4>(c0, c, s, (T)0, gx, gy, gz, gm);
      c1[2] = make_vec(c1[2], (T)-1);
      c1[3] = make_vec(c1[3], (T)-1);
      apply_dt<T, 4>(c1, c, s, (T)0, gx, gy, gz, gm);
      const T sg = ta.odd ? (T)-1 : (T)1;
      c1[0] = make_vec(c1[0], sg);
      c1[1] = make_vec(c1[1], sg);
      c1[2] = make_vec(c1[2], -sg);
      c1[3] = make_vec(c1[3], -sg);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      V s0, d, s1;
      s0.x = c0[q].x + c1[q].x;
      s0.y = c0[q].y + c1[q].y;
      d.x = c0[q].x - c1[q].x;
      d.y = c0[q].y - c1[q].y;
      s1.x = ar * d.x - ai * d.y;
      s1.y = ar * d.y + ai * d.x;
      v[q] = make_vec(s0, scale);
      v[4 + q] = make_vec(s1, scale);
    }
  }
}

__device__ __forceinline__ int planes_of(int dim) { return dim == 1 ? 2 : (dim == 2 ? 4 : 8); }

// Particle-weight sums of the spectral values v of storage position (x, y, z) (v as in
// evolve_point): acc[0] += sum |c|^2, acc[1] += sum c^dag G^ c over the wave vector(s).
// (A: the accumulator type; complex64 callers sum a few points in FP32 and move the sums
// to FP64 afterwards, since every FP64 operation costs ~64 FP32 ones here)
template <typename T, typename A>
__device__ __forceinline__ void weights_point(int dim, const AxesDev& a, int64_t x, int64_t y, int64_t z,
                                              const Mass& ms, const typename Cx2<T>::t (&vin)[8], A (&acc)[2]) {
  using V = typename Cx2<T>::t;
  int64_t f[3], fs;
  wave_vectors(dim, x, y, z, a, f, fs);
  const int S = dim == 1 ? 2 : 4;
  const int nq = dim == 3 ? 2 : 1;
  V vq[2][4];
  if (dim == 3) {
    T ar, ai;
    coset_phase_tab<T>(a, f, ar, ai);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const V p0 = vin[q], p1 = vin[4 + q];
      V b;
      b.x = ar * p1.x + ai * p1.y;
      b.y = ar * p1.y - ai * p1.x;
      vq[0][q].x = p0.x + b.x;
      vq[0][q].y = p0.y + b.y;
      vq[1][q].x = p0.x - b.x;
      vq[1][q].y = p0.y - b.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) vq[0][q] = vin[q];
  }
  // G^ of the BCC half spectrum q1 is -Gamma G^_q0 Gamma (Gamma = diag(I, -I); see
  // evolve_point): v^dag G^_q1 v = -(Gamma v)^dag G^_q0 (Gamma v)
  T gx, gy, gz, gm;
  ghat<T>(dim, a, f, 0, ms, gx, gy, gz, gm);
  if (dim == 3) {
    vq[1][2] = make_vec(vq[1][2], (T)-1);
    vq[1][3] = make_vec(vq[1][3], (T)-1);
  }
  for (int j = 0; j < nq; ++j) {
    // cos = 1, sin = 1 turns apply_dt into v - i G^ v; recover G^ v from it
    T nrm = 0, gdot = 0;
    if (S == 2) {
      V v[2] = {vq[j][0], vq[j][1]};
      V w[2] = {v[0], v[1]};
      apply_dt<T, 2>(w, (T)0, (T)1, (T)0, gx, gy, gz, gm);  // w = -i G^ v
      for (int q = 0; q < 2; ++q) {
        nrm += v[q].x * v[q].x + v[q].y * v[q].y;
        // v^dag (G^ v) = v^dag (i w)
        gdot += -(v[q].x * w[q].y - v[q].y * w[q].x);
      }
    } else {
      V v[4] = {vq[j][0], vq[j][1], vq[j][2], vq[j][3]};
      V w[4] = {v[0], v[1], v[2], v[3]};
      apply_dt<T, 4>(w, (T)0, (T)1, (T)0, gx, gy, gz, gm);
      for (int q = 0; q < 4; ++q) {
        nrm += v[q].x * v[q].x + v[q].y * v[q].y;
        gdot += -(v[q].x * w[q].y - v[q].y * w[q].x);
      }
    }
    acc[0] += (A)nrm;
    acc[1] += j ? -(A)gdot : (A)gdot;
  }
}

// Byte offset of the row constants after the L x CP line buffer (16-byte aligned).
__host__ __device__ constexpr size_t fused_rowc_offset(int L, int CP) {
  return (((size_t)L * CP * sizeof(float2)) + 15) & ~size_t(15);
}

// Row constants of the BCC symbol for the fused x pass.  With (cy, sy), (cz, sz) the
// half-angle table entries of a row's y and z frequencies, A = cy cz, B = sy sz,
// Cc = sy cz, D = cy sz give, for the x entry (cx, sx) of wave vector q0,
//   n~ = (sx A - cx B, cx Cc + sx D, cx D - sx Cc)   (u = cx A + sx B is not needed: the
// phase comes from the table), and the coset phase a = (cx + i sx)((A - B) + i (D + Cc)).
__device__ __forceinline__ float4 bcc_row_consts(const AxesDev& a, int64_t row) {
  const int ny = (int)a.len[1], rowi = (int)row;  // rows per plane < 2^31
  const int64_t fy = freq_of(rowi % ny, a, 1), fz = freq_of(rowi / ny, a, 2);
  float cy, sy, cz, sz;
  tab<float>(a, 1, fy, cy, sy);
  tab<float>(a, 2, fz, cz, sz);
  return make_float4(cy * cz, sy * sz, sy * cz, cy * sz);
}

// evolve_point for a BCC cell in complex64 from its row constants rc and x frequency k
// (the table slot of q0 is slot): G^ from an FP32 reciprocal square root with one Newton
// step, and the scale, the halves of the coset mix and (-1)^t folded into cos and sin.
__device__ __forceinline__ void evolve_bcc_row(const AxesDev& a, int k, float4 rc, const Mass& ms,
                                               const float2* __restrict__ nu_tab, int64_t slot,
                                               const TimeArg& ta, float scale, float2 (&v)[8]) {
  using V = float2;
  float cx, sx;
  tab<float>(a, 0, k, cx, sx);
  const float nx = sx * rc.x - cx * rc.y, ny = cx * rc.z + sx * rc.w, nz = cx * rc.w - sx * rc.z;
  const float S2 = fmaf(ms.nf * ms.nf, fmaf(nx, nx, fmaf(ny, ny, nz * nz)), ms.mf * ms.mf);  // sin^2 omega
  float inv = 0.f;
  if (S2 > 0.f) {
    const float r = rsqrtf(S2);
    inv = r * fmaf(-0.5f * S2 * r, r, 1.5f);
  }
  const float ni = ms.nf * inv;
  const float gx = ni * nx, gy = ni * ny, gz = ni * nz, gm = ms.mf * inv;
  const float pr = rc.x - rc.y, pim = rc.w + rc.z;
  const float ar = cx * pr - sx * pim, ai = cx * pim + sx * pr;  // a = exp(i (k1 + k2 + k3) / 2)
  float c, s;
  const float2 nu = nu_tab[slot];
  if (ta.small) {
    phase_split(nu, ta.tf, c, s);
  } else {
    cs_of<float, 4>(6.283185307179586232 * ((double)nu.x + (double)nu.y), ta.tt, c, s);
  }
  const float hs = 0.5f * scale;
  c *= hs;
  s *= hs;
  // c0 = Psi0 + a* Psi1, and Gamma c1 with c1 = Psi0 - a* Psi1 (the halves are in hs)
  V c0[4], c1[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    V b;
    b.x = ar * v[4 + q].x + ai * v[4 + q].y;
    b.y = ar * v[4 + q].y - ai * v[4 + q].x;
    c0[q].x = v[q].x + b.x;
    c0[q].y = v[q].y + b.y;
    c1[q].x = q < 2 ? v[q].x - b.x : b.x - v[q].x;
    c1[q].y = q < 2 ? v[q].y - b.y : b.y - v[q].y;
  }
  // D_q0^t c0 and D_q1^t c1 = (-1)^t Gamma D_q0^t (Gamma c1)
  apply_dt<float, 4>(c0, c, s, 0.f, gx, gy, gz, gm);
  const float sg = ta.odd ? -1.f : 1.f;
  apply_dt<float, 4>(c1, sg * c, sg * s, 0.f, gx, gy, gz, gm);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float ex = q < 2 ? c1[q].x : -c1[q].x, ey = q < 2 ? c1[q].y : -c1[q].y;  // Gamma
    const float dx = c0[q].x - ex, dy = c0[q].y - ey;
    v[q].x = c0[q].x + ex;
    v[q].y = c0[q].y + ey;
    v[4 + q].x = ar * dx - ai * dy;
    v[4 + q].y = ar * dy + ai * dx;
  }
}

// weights_point for a BCC cell in complex64 from its row constants rc and x frequency k
// (G^ as in evolve_bcc_row): acc[0] += |c0|^2 + |c1|^2, acc[1] += c0^dag G^_q0 c0 +
// c1^dag G^_q1 c1 with G^_q1 = -Gamma G^_q0 Gamma.
__device__ __forceinline__ void weights_bcc_row(const AxesDev& a, int k, float4 rc, const Mass& ms,
                                                const float2 (&v)[8], float (&acc)[2]) {
  using V = float2;
  float cx, sx;
  tab<float>(a, 0, k, cx, sx);
  const float nx = sx * rc.x - cx * rc.y, ny = cx * rc.z + sx * rc.w, nz = cx * rc.w - sx * rc.z;
  const float S2 = fmaf(ms.nf * ms.nf, fmaf(nx, nx, fmaf(ny, ny, nz * nz)), ms.mf * ms.mf);
  float inv = 0.f;
  if (S2 > 0.f) {
    const float r = rsqrtf(S2);
    inv = r * fmaf(-0.5f * S2 * r, r, 1.5f);
  }
  const float ni = ms.nf * inv;
  const float gx = ni * nx, gy = ni * ny, gz = ni * nz, gm = ms.mf * inv;
  const float pr = rc.x - rc.y, pim = rc.w + rc.z;
  const float ar = cx * pr - sx * pim, ai = cx * pim + sx * pr;
  V c0[4], c1[4];  // c0 = Psi0 + a* Psi1 and Gamma c1, c1 = Psi0 - a* Psi1
  float nrm = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    V b;
    b.x = ar * v[4 + q].x + ai * v[4 + q].y;
    b.y = ar * v[4 + q].y - ai * v[4 + q].x;
    c0[q].x = v[q].x + b.x;
    c0[q].y = v[q].y + b.y;
    c1[q].x = q < 2 ? v[q].x - b.x : b.x - v[q].x;
    c1[q].y = q < 2 ? v[q].y - b.y : b.y - v[q].y;
    nrm += c0[q].x * c0[q].x + c0[q].y * c0[q].y + c1[q].x * c1[q].x + c1[q].y * c1[q].y;
  }
  V w0[4], w1[4];
  ghat_mul<float, 4>(c0, gx, gy, gz, gm, w0);
  ghat_mul<float, 4>(c1, gx, gy, gz, gm, w1);
  float g = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    g += (c0[q].x * w0[q].x + c0[q].y * w0[q].y) - (c1[q].x * w1[q].x + c1[q].y * w1[q].y);
  acc[0] += nrm;
  acc[1] += g;
}

// Fused x pass of the Fourier form (complex64): for RW rows of every component
// plane, the forward DFT along x, D_k^t per wave vector (BCC coset mix included)
// and the inverse DFT along x, with one read and one write of those rows.  The y
// and z transforms run as ordinary passes before and after (transforms along
// different axes commute).  Needs the x axis in one register pass of length
// L = R1 * R2 (natural order along x); y, z may be digit-permuted (freq_of).
template <int R1, int R2>
__global__ void __launch_bounds__(256, 3) fused_x_kernel(int dim, AxesDev a, int64_t count, Mass ms,
                                                      const double* __restrict__ omega, TimeArg ta, float scale_in,
                                                      const double* __restrict__ norm0, float2* __restrict__ data,
                                                      const float2* __restrict__ tw_line) {
  using V = float2;
  constexpr int L = R1 * R2, TPL = R1 > R2 ? R1 : R2, C = 256 / TPL;
  constexpr int CP = (C % 2 == 0) ? C + 1 : C;
  extern __shared__ __align__(16) unsigned char fx_smem[];
  V* sm = reinterpret_cast<V*>(fx_smem);
  float4* rowc = reinterpret_cast<float4*>(fx_smem + fused_rowc_offset(L, CP));  // BCC row constants
  const float scale = norm0 ? scale_in * rsqrtf((float)norm0[0]) : scale_in;
  const int P = planes_of(dim);
  const int RW = C / P;                     // rows per CTA (C >= 8 >= P)
  const int CU = RW * P;                    // lines in use
  const int64_t nrows = count / L;          // rows per plane
  const int64_t row0 = (int64_t)blockIdx.x * RW;
  const bool bcc_rows = dim == 3 && omega != nullptr;
  const int tid = threadIdx.x, c = tid % C, r = tid / C;
  const TwRow<V> tw{tw_line, r};
  // ---- load (cp.async): consecutive threads read consecutive x of one line; line cc = w P + p
  // holds plane p of row row0 + w (P is a power of two).  Element e = tid + 256 j sits
  // at line e / L, position e % L, from tid / L and tid % L plus compile-time offsets.
  constexpr int NE = (C * L + 255) / 256;
  const int t_c = tid / L, t_x = tid - (tid / L) * L;
  const int lgP = dim == 1 ? 1 : (dim == 2 ? 2 : 3);
#pragma unroll
  for (int j = 0; j < NE; ++j) {
    int xx = t_x + (256 * j) % L, cc = t_c + (256 * j) / L;
    if (xx >= L) {
      xx -= L;
      ++cc;
    }
    const int p = cc & (P - 1), w = cc >> lgP;
    const bool ok = cc < CU && row0 + w < nrows;
    if (cc < C) cp_async_elem(&sm[cc + CP * xx], ok ? data + p * count + (row0 + w) * L + xx : data, ok);
  }
  if (bcc_rows && tid < RW && row0 + tid < nrows) rowc[tid] = bcc_row_consts(a, row0 + tid);  // while loading
  cp_async_wait_all();
  __syncthreads();
  reg_fft_steps<float, false, R1, R2, CP>(sm, c, r, tw);
  // ---- D_k^t at every (row, k) of the CTA
  if (bcc_rows) {
    const float2* nu_tab = reinterpret_cast<const float2*>(omega);
    for (int q = tid; q < RW * L; q += 256) {
      const int w = q / L, k = q - w * L;
      const int64_t row = row0 + w;
      if (row >= nrows) continue;
      V v[8];
#pragma unroll
      for (int pp = 0; pp < 8; ++pp) v[pp] = sm[w * 8 + pp + CP * k];
      evolve_bcc_row(a, k, rowc[w], ms, nu_tab, row * L + k, ta, scale, v);
#pragma unroll
      for (int pp = 0; pp < 8; ++pp) sm[w * 8 + pp + CP * k] = v[pp];
    }
  } else {
    for (int q = tid; q < RW * L; q += 256) {
      const int w = q / L, k = q - w * L;
      const int64_t row = row0 + w;
      if (row >= nrows) continue;
      const int ny = (int)a.len[1], rowi = (int)row;  // rows per plane < 2^31
      const int64_t yy = rowi % ny, zz = rowi / ny;
      V v[8];
#pragma unroll
      for (int pp = 0; pp < 8; ++pp)
        if (pp < P) v[pp] = sm[w * P + pp + CP * k];
      evolve_point<float>(dim, a, k, yy, zz, row * L + k, ms, omega, ta, scale, v);
#pragma unroll
      for (int pp = 0; pp < 8; ++pp)
        if (pp < P) sm[w * P + pp + CP * k] = v[pp];
    }
  }
  __syncthreads();
  reg_fft_steps<float, true, R1, R2, CP>(sm, c, r, tw);
  // ---- store
#pragma unroll
  for (int j = 0; j < NE; ++j) {
    int xx = t_x + (256 * j) % L, cc = t_c + (256 * j) / L;
    if (xx >= L) {
      xx -= L;
      ++cc;
    }
    const int p = cc & (P - 1), w = cc >> lgP;
    if (cc < CU && row0 + w < nrows) data[p * count + (row0 + w) * L + xx] = sm[cc + CP * xx];
  }
}

template <int R1, int R2>
qw_status launch_fused(const Geometry& g, const SpecAxes& ax, double n, double m, const double* omega,
                              int64_t t, void* psi, const void* tw_line, cudaStream_t st, const double* norm0) {
  constexpr int L = R1 * R2, TPL = R1 > R2 ? R1 : R2, C = 256 / TPL;
  constexpr int CP = (C % 2 == 0) ? C + 1 : C;
  const int P = g.dim == 1 ? 2 : (g.dim == 2 ? 4 : 8);
  const int RW = C / P;
  const int64_t nrows = g.vol / L;
  const int64_t grid = (nrows + RW - 1) / RW;
  const size_t smem = fused_rowc_offset(L, CP) + 8 * sizeof(float4);  // lines, then up to 8 row constants
  const qw_status sa = smem_attr(fused_x_kernel<R1, R2>, (int)smem);
  if (sa != QW_OK) return sa;
  fused_x_kernel<R1, R2><<<(unsigned)grid, 256, smem, st>>>(
      g.dim, to_dev(ax), g.vol, make_mass(n, m), omega, make_time(t), (float)(1.0 / (double)g.vol), norm0,
      static_cast<float2*>(psi), static_cast<const float2*>(tw_line));
  QW_CHECK_LAUNCH("fused x pass launch");
  return QW_OK;
}

// Particle-weight sums of a spectrum whose remaining transform is the x DFT (complex64):
// the rows of every plane (already transformed along y and z) come in by cp.async, are
// transformed along x in shared memory and summed per wave vector (weights_point); nothing
// is written back.  Same tiling as fused_x_kernel; partials[2 b], [2 b + 1] per CTA b.
template <int R1, int R2>
__global__ void __launch_bounds__(256, 3) weights_x_kernel(int dim, AxesDev a, int64_t count, Mass ms,
                                                        const float2* __restrict__ data,
                                                        const float2* __restrict__ tw_line,
                                                        double* __restrict__ partials) {
  using V = float2;
  constexpr int L = R1 * R2, TPL = R1 > R2 ? R1 : R2, C = 256 / TPL;
  constexpr int CP = (C % 2 == 0) ? C + 1 : C;
  extern __shared__ __align__(16) unsigned char wx_smem[];
  V* sm = reinterpret_cast<V*>(wx_smem);
  float4* rowc = reinterpret_cast<float4*>(wx_smem + fused_rowc_offset(L, CP));  // BCC row constants
  const int P = planes_of(dim);
  const int RW = C / P, CU = RW * P;
  const int64_t nrows = count / L;
  const int64_t row0 = (int64_t)blockIdx.x * RW;
  const int tid = threadIdx.x, c = tid % C, r = tid / C;
  const TwRow<V> tw{tw_line, r};
  constexpr int NE = (C * L + 255) / 256;
  const int t_c = tid / L, t_x = tid - (tid / L) * L;
  const int lgP = dim == 1 ? 1 : (dim == 2 ? 2 : 3);
#pragma unroll
  for (int j = 0; j < NE; ++j) {
    int xx = t_x + (256 * j) % L, cc = t_c + (256 * j) / L;
    if (xx >= L) {
      xx -= L;
      ++cc;
    }
    const int p = cc & (P - 1), w = cc >> lgP;
    const bool ok = cc < CU && row0 + w < nrows;
    if (cc < C) cp_async_elem(&sm[cc + CP * xx], ok ? data + p * count + (row0 + w) * L + xx : data, ok);
  }
  if (dim == 3 && tid < RW && row0 + tid < nrows) rowc[tid] = bcc_row_consts(a, row0 + tid);  // while loading
  cp_async_wait_all();
  __syncthreads();
  reg_fft_steps<float, false, R1, R2, CP>(sm, c, r, tw);
  float facc[2] = {0.f, 0.f};  // a thread sums RW L / 256 points (2-4) in FP32
  if (dim == 3) {
    for (int q = tid; q < RW * L; q += 256) {
      const int w = q / L, k = q - w * L;
      if (row0 + w >= nrows) continue;
      V v[8];
#pragma unroll
      for (int pp = 0; pp < 8; ++pp) v[pp] = sm[w * 8 + pp + CP * k];
      weights_bcc_row(a, k, rowc[w], ms, v, facc);
    }
  } else {
    for (int q = tid; q < RW * L; q += 256) {
      const int w = q / L, k = q - w * L;
      const int64_t row = row0 + w;
      if (row >= nrows) continue;
      const int ny = (int)a.len[1], rowi = (int)row;
      const int64_t yy = rowi % ny, zz = rowi / ny;
      V v[8];
#pragma unroll
      for (int pp = 0; pp < 8; ++pp)
        if (pp < P) v[pp] = sm[w * P + pp + CP * k];
      weights_point<float>(dim, a, k, yy, zz, ms, v, facc);
    }
  }
  // warp sums in FP32 (64 points), the eight warp sums in FP64 in a fixed order: an FP64
  // block reduction per thread would cost more than the thread's points here
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    facc[0] += __shfl_xor_sync(0xffffffffu, facc[0], o);
    facc[1] += __shfl_xor_sync(0xffffffffu, facc[1], o);
  }
  __shared__ float wsum[8][2];
  if ((tid & 31) == 0) {
    wsum[tid >> 5][0] = facc[0];
    wsum[tid >> 5][1] = facc[1];
  }
  __syncthreads();
  if (tid == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int w = 0; w < 8; ++w) {
      a0 += (double)wsum[w][0];
      a1 += (double)wsum[w][1];
    }
    partials[2 * blockIdx.x] = a0;
    partials[2 * blockIdx.x + 1] = a1;
  }
}

// CTAs of the fused x pass and of weights_x_kernel (rows of RW per CTA)
template <int R1, int R2>
inline int64_t fused_x_ctas(const Geometry& g) {
  constexpr int TPL = R1 > R2 ? R1 : R2, C = 256 / TPL;
  const int RW = C / (g.dim == 1 ? 2 : (g.dim == 2 ? 4 : 8));
  return (g.vol / g.nx + RW - 1) / RW;
}

template <int R1, int R2>
qw_status launch_weights_x(const Geometry& g, const SpecAxes& ax, double n, double m, const void* data,
                           const void* tw_line, double* partials, cudaStream_t st) {
  constexpr int L = R1 * R2, TPL = R1 > R2 ? R1 : R2, C = 256 / TPL;
  constexpr int CP = (C % 2 == 0) ? C + 1 : C;
  const size_t smem = fused_rowc_offset(L, CP) + 8 * sizeof(float4);  // lines, then up to 8 row constants
  const qw_status sa = smem_attr(weights_x_kernel<R1, R2>, (int)smem);
  if (sa != QW_OK) return sa;
  weights_x_kernel<R1, R2><<<(unsigned)fused_x_ctas<R1, R2>(g), 256, smem, st>>>(
      g.dim, to_dev(ax), g.vol, make_mass(n, m), static_cast<const float2*>(data),
      static_cast<const float2*>(tw_line), partials);
  QW_CHECK_LAUNCH("x-pass particle weights launch");
  return QW_OK;
}

// Line lengths of the fused x pass: the register lengths from 64 up (shorter x axes are
// small boxes, where the separate passes cost as little), in six groups that the
// instantiation units fused_x_[1-6].cu compile in parallel.
#define QW_FUSED_LENGTHS_1(X) X(64, 8, 8) X(72, 9, 8) X(81, 9, 9)
#define QW_FUSED_LENGTHS_2(X) X(96, 12, 8) X(108, 12, 9) X(128, 16, 8)
#define QW_FUSED_LENGTHS_3(X) X(144, 12, 12) X(162, 18, 9) X(192, 16, 12)
#define QW_FUSED_LENGTHS_4(X) X(216, 18, 12) X(243, 27, 9)
#define QW_FUSED_LENGTHS_5(X) X(256, 16, 16) X(288, 18, 16) X(324, 18, 18)
#define QW_FUSED_LENGTHS_6(X) X(384, 24, 16) X(432, 24, 18) X(512, 32, 16)
#define QW_FUSED_LENGTHS(X)                                                                       \
  QW_FUSED_LENGTHS_1(X) QW_FUSED_LENGTHS_2(X) QW_FUSED_LENGTHS_3(X) QW_FUSED_LENGTHS_4(X) \
  QW_FUSED_LENGTHS_5(X) QW_FUSED_LENGTHS_6(X)
#define QW_FUSED_X_INSTANTIATE(LEN, A, B)                                                                     \
  template qw_status launch_fused<A, B>(const Geometry&, const SpecAxes&, double, double, const double*,  \
                                        int64_t, void*, const void*, cudaStream_t, const double*);         \
  template qw_status launch_weights_x<A, B>(const Geometry&, const SpecAxes&, double, double, const void*, \
                                            const void*, double*, cudaStream_t);
#define QW_FUSED_X_EXTERN(LEN, A, B)                                                                               \
  extern template qw_status launch_fused<A, B>(const Geometry&, const SpecAxes&, double, double, const double*,  \
                                               int64_t, void*, const void*, cudaStream_t, const double*);         \
  extern template qw_status launch_weights_x<A, B>(const Geometry&, const SpecAxes&, double, double, const void*, \
                                                   const void*, double*, cudaStream_t);

}  // namespace qw
