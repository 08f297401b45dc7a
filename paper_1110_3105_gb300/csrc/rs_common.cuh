// Shared device/host definitions for the recursive-skeletonization library.
//
// Scalar types: the real kernels (2D/3D Laplace) run in double (build) and
// float (mixed-precision solve); the Helmholtz kernels (2D and 3D) in
// complex<double> and complex<float>; double-float pairs (and complex pairs
// of them) carry the refinement residual.  The complex type is a plain two-field struct with the
// operators the kernels need, interleaved (re, im) like C99 double complex.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include <string>

#include "../../include/rs.h"

namespace rs {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
int fail(int code, const char* fmt, ...);

#define RS_CUDA(call)                                                          \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      cudaGetLastError(); /* do not leak a non-sticky error into later calls */ \
      return ::rs::fail(RS_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call, \
                        cudaGetErrorString(e_));                               \
    }                                                                          \
  } while (0)

// Every kernel launch of the library is followed by RS_CHECK_LAUNCH(), which
// also counts it (rs_launch_count()).
void count_launch();
#define RS_CHECK_LAUNCH()  \
  do {                     \
    ::rs::count_launch();  \
    RS_CUDA(cudaGetLastError()); \
  } while (0)

#define RS_TRY(expr)            \
  do {                          \
    int rc_ = (expr);           \
    if (rc_ != RS_OK) return rc_; \
  } while (0)

// ------------------------------------------------------------ complex type
template <class R>
struct cplx {
  R re, im;
  cplx() = default;
  __host__ __device__ cplx(R r) : re(r), im(0) {}
  __host__ __device__ cplx(R r, R i) : re(r), im(i) {}
  template <class Q>
  __host__ __device__ explicit cplx(const cplx<Q>& o) : re((R)o.re), im((R)o.im) {}
};
template <class R> __host__ __device__ inline cplx<R> operator+(cplx<R> a, cplx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R> __host__ __device__ inline cplx<R> operator-(cplx<R> a, cplx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R> __host__ __device__ inline cplx<R> operator-(cplx<R> a) { return {-a.re, -a.im}; }
template <class R> __host__ __device__ inline cplx<R> operator*(cplx<R> a, cplx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R> __host__ __device__ inline cplx<R> operator*(R s, cplx<R> a) { return {s * a.re, s * a.im}; }
template <class R> __host__ __device__ inline cplx<R>& operator+=(cplx<R>& a, cplx<R> b) { a.re += b.re; a.im += b.im; return a; }
template <class R> __host__ __device__ inline cplx<R>& operator-=(cplx<R>& a, cplx<R> b) { a.re -= b.re; a.im -= b.im; return a; }
template <class R> __host__ __device__ inline cplx<R> operator/(cplx<R> a, cplx<R> b) {
  R d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
template <class R> __host__ __device__ inline bool operator==(cplx<R> a, cplx<R> b) { return a.re == b.re && a.im == b.im; }

using c64 = cplx<float>;
using c128 = cplx<double>;

// Generic scalar helpers -----------------------------------------------------
__host__ __device__ inline double abs2(double x) { return x * x; }
__host__ __device__ inline float abs2(float x) { return x * x; }
template <class R> __host__ __device__ inline R abs2(cplx<R> z) { return z.re * z.re + z.im * z.im; }
__host__ __device__ inline double conj_(double x) { return x; }
__host__ __device__ inline float conj_(float x) { return x; }
template <class R> __host__ __device__ inline cplx<R> conj_(cplx<R> z) { return {z.re, -z.im}; }
__host__ __device__ inline double real_(double x) { return x; }
template <class R> __host__ __device__ inline R real_(cplx<R> z) { return z.re; }

template <class S> struct real_of { using type = S; };
template <class R> struct real_of<cplx<R>> { using type = R; };
template <class S> struct lowp { using type = float; };
template <> struct lowp<c128> { using type = c64; };
template <class S> struct is_cplx { static constexpr bool value = false; };
template <class R> struct is_cplx<cplx<R>> { static constexpr bool value = true; };

template <class S> __device__ inline S shfl_xor(S v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
template <class R> __device__ inline cplx<R> shfl_xor(cplx<R> v, int m) {
  return {__shfl_xor_sync(0xffffffffu, v.re, m), __shfl_xor_sync(0xffffffffu, v.im, m)};
}
template <class S> __device__ inline S shfl(S v, int src) { return __shfl_sync(0xffffffffu, v, src); }
template <class R> __device__ inline cplx<R> shfl(cplx<R> v, int src) {
  return {__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src)};
}
template <class S> __device__ inline S warp_sum(S v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
  return v;
}
// Sum over aligned groups of G lanes (G a power of two <= 32); every lane of
// a group gets its group's sum.  All 32 lanes must take part.
template <int G, class S> __device__ inline S group_sum(S v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += shfl_xor(v, o);
  return v;
}

// ----------------------------------------------------------- point clouds
// Points are stored per axis (structure of arrays) in tree order.
struct Pts {
  const double* x;
  const double* y;
  const double* z;  // null in 2D
  // outward unit normals and curvature (double-layer kernel only, else null)
  const double* nx;
  const double* ny;
  const double* kap;
};

__device__ inline double dist2(const Pts& p, int i, int j) {
  double dx = p.x[i] - p.x[j], dy = p.y[i] - p.y[j];
  double s = dx * dx + dy * dy;
  if (p.z) { double dz = p.z[i] - p.z[j]; s += dz * dz; }
  return s;
}
__device__ inline double dist(const Pts& p, int i, int j) { return sqrt(dist2(p, i, j)); }

// Kernel parameters shared by every device routine.
struct KParams {
  int kind;       // RS_LAPLACE2D / RS_HELMHOLTZ2D / RS_LAPLACE3D / RS_HELMHOLTZ3D
  double w;       // quadrature weight in A = I + w K
  double kwave;   // Helmholtz wavenumber
  const double* logtab;   // device table of log_tab (see below)
};

// Natural logarithm by Tang's table-driven method (P. T. P. Tang, "Table-
// driven implementation of the logarithm function in IEEE floating-point
// arithmetic", ACM TOMS 16(4), 1990): x = 2^e m with m in [1, 2); c = 1 +
// i/256 from the top 8 bits of m; log x = e log 2 + log c + log(1 + t) with
// t = m/c - 1 in [0, 1/256), the last by its Taylor series to t^7 (remainder
// < 2e-19).  The table holds (log c_i, 1/c_i) pairs and, last, log 2 split
// into a 32-bit head (so e * head is exact) and the rest, all computed on the
// host in extended precision.  About 11 FP64 operations against ~25 of the general
// routine; the error stays within a few units of 1e-16 absolute.  Inputs
// outside the positive normal range take the library log.
constexpr int LOGTAB_N = 256;
__device__ __forceinline__ double log_tab(const double* tab, double x) {
  const int hi = __double2hiint(x);
  const int e = (hi >> 20) - 1023;
  if (hi <= 0x000FFFFF || hi >= 0x7FF00000) return log(x);   // zero, subnormal, negative, inf, nan
  const int i = (hi >> 12) & 0xFF;
  const double m = __hiloint2double((hi & 0x000FFFFF) | 0x3FF00000, __double2loint(x));
  const double2 li = __ldg(reinterpret_cast<const double2*>(tab) + i);   // (log c_i, 1 / c_i)
  const double t = fma(m, li.y, -1.0);
  double q = 1.0 / 7.0;
  q = fma(q, t, -1.0 / 6.0);
  q = fma(q, t, 1.0 / 5.0);
  q = fma(q, t, -1.0 / 4.0);
  q = fma(q, t, 1.0 / 3.0);
  q = fma(q, t, -0.5);
  const double l1p = fma(q * t, t, t);   // t + t^2 q(t)
  const double2 ln2 = __ldg(reinterpret_cast<const double2*>(tab) + LOGTAB_N);
  return fma((double)e, ln2.x, li.x + fma((double)e, ln2.y, l1p));
}

// Green's functions: eq. 2d-laplace, eq. 3d-laplace, eq. 2d-helmholtz,
// eq. 3d-helmholtz.  H0^(1) = J0 + i Y0, cos and sin from CUDA's math library.
__device__ inline double green_real(int kind, double r) {
  if (kind == RS_LAPLACE3D) return 1.0 / (4.0 * M_PI * r);
  return -log(r) * (1.0 / (2.0 * M_PI));
}
// The same from the squared distance s = r^2 (no square root on the FP64
// pipe: log r = log(s) / 2, 1 / r = rsqrt(s)).
__device__ inline double green_real_s2(const KParams& kp, double s) {
  if (kp.kind == RS_LAPLACE3D) return rsqrt(s) * (1.0 / (4.0 * M_PI));
  return -log_tab(kp.logtab, s) * (1.0 / (4.0 * M_PI));
}
__device__ inline c128 green_cplx(int kind, double kwave, double r) {
  const double kr = kwave * r;
  if (kind == RS_HELMHOLTZ3D) {   // e^{i k r} / (4 pi r)
    double s, c;
    sincos(kr, &s, &c);
    const double f = 1.0 / (4.0 * M_PI * r);
    return c128(c * f, s * f);
  }
  return c128(-0.25 * y0(kr), 0.25 * j0(kr));   // (i/4)(J0 + i Y0)
}
// Double-layer kernel dG/dnu_y (x, y) for the 2D Laplace G (eq. double-layer):
// (1/2 pi) (x - y) . nu_y / |x - y|^2, target x = (tx, ty), source j.
__device__ inline double dlayer_at(const Pts& p, double tx, double ty, int j) {
  const double dx = tx - p.x[j], dy = ty - p.y[j];
  return (dx * p.nx[j] + dy * p.ny[j]) / (2.0 * M_PI * (dx * dx + dy * dy));
}
// w K(x_i, x_j) for distinct points: target i, source j.
template <class S> __device__ inline S offdiag_entry(const KParams& kp, const Pts& p, int i, int j);
template <> __device__ inline double offdiag_entry<double>(const KParams& kp, const Pts& p, int i, int j) {
  if (kp.kind == RS_LAPLACE2D_DL) return kp.w * dlayer_at(p, p.x[i], p.y[i], j);
  return kp.w * green_real_s2(kp, dist2(p, i, j));
}
template <> __device__ inline c128 offdiag_entry<c128>(const KParams& kp, const Pts& p, int i, int j) {
  c128 g = green_cplx(kp.kind, kp.kwave, dist(p, i, j));
  return c128(kp.w * g.re, kp.w * g.im);
}
// A_ij = delta_ij + w K(x_i, x_j) with K_ii = 0; for the double layer K_ii
// is the kernel's limit on a smooth curve, -kappa_i / (4 pi).
template <class S> __device__ inline S system_entry(const KParams& kp, const Pts& p, int i, int j) {
  if (i == j) return kp.kind == RS_LAPLACE2D_DL ? S(1.0 - kp.w * p.kap[i] * (0.25 / M_PI)) : S(1.0);
  return offdiag_entry<S>(kp, p, i, j);
}

// Green's function between an arbitrary location and a point.
template <class S> __device__ inline S green_at(const KParams& kp, double r);
template <> __device__ inline double green_at<double>(const KParams& kp, double r) { return kp.w * green_real(kp.kind, r); }
template <> __device__ inline c128 green_at<c128>(const KParams& kp, double r) {
  c128 g = green_cplx(kp.kind, kp.kwave, r);
  return c128(kp.w * g.re, kp.w * g.im);
}
// The same from the squared distance.
template <class S> __device__ inline S green_at_s2(const KParams& kp, double s);
template <> __device__ inline double green_at_s2<double>(const KParams& kp, double s) {
  return kp.w * green_real_s2(kp, s);
}
template <> __device__ inline c128 green_at_s2<c128>(const KParams& kp, double s) { return green_at<c128>(kp, sqrt(s)); }

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ------------------------------------------------------------ double-float
// An unevaluated sum hi + lo of two floats (about 48 significant bits).
// Products use the exact FMA two-product, sums the exact two-sum (Dekker
// 1971; Knuth, TAOCP vol. 2, Sec. 4.2.2); every operation is explicitly
// rounded so the compiler cannot fuse a product into a following sum.
struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ dfloat(float h, float l) : hi(h), lo(l) {}
  __device__ explicit dfloat(double x) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(__dsub_rn(x, (double)hi));
  }
};
__device__ __forceinline__ dfloat df_renorm(dfloat s) {
  float t = __fadd_rn(s.hi, s.lo);
  return dfloat(t, __fsub_rn(s.lo, __fsub_rn(t, s.hi)));
}
// s += a * b
__device__ __forceinline__ void df_fma(dfloat& s, dfloat a, dfloat b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float t = __fadd_rn(s.hi, p);
  float bb = __fsub_rn(t, s.hi);
  float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  s.lo = __fadd_rn(s.lo, __fadd_rn(err, e));
  s.hi = t;
}
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  float t = __fadd_rn(a.hi, b.hi);
  float bb = __fsub_rn(t, a.hi);
  float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(t, bb)), __fsub_rn(b.hi, bb));
  return df_renorm(dfloat(t, __fadd_rn(a.lo, __fadd_rn(err, b.lo))));
}

// Complex double-float: real and imaginary parts each a double-float.
struct cdfloat {
  dfloat re, im;
  cdfloat() = default;
  __host__ __device__ cdfloat(dfloat r, dfloat i) : re(r), im(i) {}
  __device__ explicit cdfloat(double x) : re(x), im(0.0f, 0.0f) {}
};
__device__ __forceinline__ cdfloat operator+(cdfloat a, cdfloat b) { return cdfloat(a.re + b.re, a.im + b.im); }
// s += a * b (four double-float products)
__device__ __forceinline__ void cdf_fma(cdfloat& s, cdfloat a, cdfloat b) {
  df_fma(s.re, a.re, b.re);
  df_fma(s.re, dfloat(-a.im.hi, -a.im.lo), b.im);
  df_fma(s.im, a.re, b.im);
  df_fma(s.im, a.im, b.re);
}


// ------------------------------------------------- conversions off the FP64 pipe
// Double <-> float conversions issue on the FP64 pipe, which on this GPU runs
// at 1/64 of the FP32 rate; in the bandwidth kernels they would cost more
// than the arithmetic.  These do the same conversions with integer
// instructions, by the IEEE-754 binary64/binary32 layouts (sign | biased
// exponent | fraction; biases 1023 and 127): round to nearest even by adding
// half an ulp (minus one, plus the kept lowest bit) before the shift.  Values
// outside the float normal range take the hardware conversion.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned int hi = (unsigned int)(u >> 32);
  const unsigned int e = (hi >> 20) & 0x7FFu;
  if (e - 897u < 253u) {   // float exponent e - 896 in [1, 253]: no overflow after a rounding carry
    const unsigned long long m = u & 0x7FFFFFFFFFFFFFFFull;
    const unsigned long long r = m + 0x0FFFFFFFull + ((m >> 29) & 1ull);
    return __uint_as_float(((unsigned int)(r >> 29) - (896u << 23)) | (hi & 0x80000000u));
  }
  return __double2float_rn(x);
}
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int mag = b & 0x7FFFFFFFu;
  if (mag - 0x00800000u < 0x7F000000u)   // normal
    return __hiloint2double((int)((b & 0x80000000u) | ((mag >> 3) + (896u << 20))), (int)(b << 29));
  if (mag == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
  return (double)f;
}
// x = hi + lo: hi is x truncated to 24 significant bits (exact), lo the
// remaining 29 bits rounded to a float (|lo| < ulp(hi), error <= 2^-24 |lo|).
__device__ __forceinline__ dfloat f64_to_df(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned int hiw = (unsigned int)(u >> 32);
  const unsigned int e = (hiw >> 20) & 0x7FFu;
  if (e - 949u < 202u) {   // both parts normal floats: e in [949, 1150]
    const unsigned int sign = hiw & 0x80000000u;
    const unsigned long long m = u & 0x7FFFFFFFFFFFFFFFull;
    const float h = __uint_as_float(((unsigned int)(m >> 29) - (896u << 23)) | sign);
    const unsigned int L = (unsigned int)m & 0x1FFFFFFFu;   // low 29 fraction bits
    // float(L) from two exact pieces (2^23 + v has v in its fraction field)
    const float lh = __uint_as_float(0x4B000000u | (L >> 6)) - 8388608.0f;
    const float ll = __uint_as_float(0x4B000000u | (L & 63u)) - 8388608.0f;
    const float lf = __fmaf_rn(lh, 64.0f, ll);
    const float scale = __uint_as_float((e - 948u) << 23);   // 2^(e - 1023 - 52)
    return dfloat(h, __uint_as_float(__float_as_uint(__fmul_rn(lf, scale)) | sign));
  }
  return dfloat(x);
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }

}  // namespace rs
