// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, giving a 48-bit significand (relative
// precision about 2^-48) on the FP32 pipes.  GB300 executes FP32 FMAs at 64x
// the FP64 rate (128 vs 2 per SM per clock), so the covariance arithmetic of
// the tracker runs faster in this form than in native FP64.
//
// Error-free transformations: TwoSum (Knuth, TAOCP vol. 2, 4.2.2),
// Fast-TwoSum (Dekker 1971, "A floating-point technique for extending the
// available precision"), TwoProd by one FMA.  Addition follows the sloppy
// renormalisation of double-double libraries (Hida, Li, Bailey 2001).  All primitive steps
// use the _rn intrinsics so the compiler neither contracts nor reorders them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tpct {

// ---------------------------------------------------------------- float <-> double on the integer pipes
// GB300 runs every FP64-pipe instruction, conversions between float and
// double included, at 2 lanes per SM per clock (1/64 of the FP32 rate).
// These two conversions rebuild the IEEE-754 bit patterns with a handful of
// integer instructions instead.  binary32 = sign | 8-bit exponent (bias 127)
// | 23-bit fraction; binary64 = sign | 11-bit exponent (bias 1023) | 52-bit
// fraction, so a normal number moves between the two by re-biasing the
// exponent (896 = 1023 - 127) and shifting the fraction by 29 bits.

// float -> double, exact for zero, normal, infinite and NaN floats; float
// subnormals (|f| < 2^-126) become zero.
__device__ __forceinline__ double widen(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t mag = b & 0x7fffffffu;
  uint32_t hi = (mag >> 3) + 0x38000000u;                  // exponent + 896 (in bits 30..20)
  uint32_t lo = b << 29;
  if (mag >= 0x7f800000u) hi = 0x7ff00000u | ((mag >> 3) & 0xfffffu);   // inf, NaN
  if (mag < 0x00800000u) { hi = 0u; lo = 0u; }              // zero, subnormal
  return __hiloint2double((int)(hi | (b & 0x80000000u)), (int)lo);
}

// double -> float, rounded to nearest (ties away from zero) by adding half a
// float ulp to the bit pattern before truncating it; results below float's
// normal range come out as zero or a subnormal below 2^-146, results above
// it saturate to a finite float within 8 ulp of the largest (the exponent
// saturates, the fraction keeps its top bits), infinities and NaNs become NaN.
__device__ __forceinline__ float narrow(double d) {
  const uint64_t u = (uint64_t)__double_as_longlong(d) + 0x10000000ull;
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  int32_t e = (int32_t)(hi & 0x7fffffffu) - 0x38000000;    // exponent - 896 (in bits 30..20)
  e = min(max(e, 0), 0x0fefffff);
  const float r = __uint_as_float((hi & 0x80000000u) | __funnelshift_l(lo, (uint32_t)e, 3));
  return (hi & 0x7ff00000u) == 0x7ff00000u ? __uint_as_float(0x7fc00000u) : r;
}

// the float/double overloads stay visible next to the df64 ones below
using ::fabs;
using ::sqrt;
using ::copysign;

struct df64 {
  float hi, lo;
  __host__ __device__ df64() : hi(0.f), lo(0.f) {}
  __host__ __device__ df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit df64(float a) : hi(a), lo(0.f) {}
  __host__ __device__ explicit df64(int a) : hi((float)a), lo(0.f) {}
  __host__ __device__ explicit df64(double a) {
#ifdef __CUDA_ARCH__
    hi = narrow(a);
    lo = narrow(a - widen(hi));
#else
    hi = (float)a;
    lo = (float)(a - (double)hi);
#endif
  }
  __host__ __device__ explicit operator float() const { return hi + lo; }
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df64 fast_two_sum(float a, float b) {   // requires |a| >= |b|
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return df64(s, e);
}

__device__ __forceinline__ df64 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df64(s, e);
}

__device__ __forceinline__ df64 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  return df64(p, e);
}

// Addition: TwoSum of the high parts, the low parts added in float, one
// renormalisation (11 instructions).  The error is bounded by ~2^-47 times
// the larger operand (not the result), like every add-then-round scheme under
// cancellation.  The only double-float user is the tracklet covariance,
// whose updates cancel by at most ~1e6 (prior variances down to cluster
// variances), which leaves ~1e-9 relative; the refit, whose diffuse prior
// amplifies rounding ~1e12, stays in native FP64.
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const df64 s = two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  df64 p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df64 operator*(df64 a, float b) {
  df64 p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df64 operator*(float b, df64 a) { return a * b; }

// a * x + y for a float a: the product's two parts feed one addition (14 instructions)
__device__ __forceinline__ df64 fma_df(float a, df64 x, df64 y) {
  df64 p = two_prod(a, x.hi);
  p.lo = __fmaf_rn(a, x.lo, p.lo);
  const df64 s = two_sum(p.hi, y.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(p.lo, y.lo));
  return fast_two_sum(s.hi, e);
}

// a / b: three float quotient digits, each the running remainder's high part
// times the float reciprocal of b's high part (the remainders correct each
// digit's error; one reciprocal instead of three IEEE divisions).
__device__ __forceinline__ df64 operator/(df64 a, df64 b) {
  const float ib = __frcp_rn(b.hi);
  const float q1 = __fmul_rn(a.hi, ib);
  df64 r = a - b * q1;
  const float q2 = __fmul_rn(r.hi, ib);
  r = r - b * q2;
  const float q3 = __fmul_rn(r.hi, ib);
  return fast_two_sum(q1, q2) + df64(q3);
}

__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { a = a + b; return a; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { a = a - b; return a; }

__device__ __forceinline__ bool operator<(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(df64 a, df64 b) { return b < a; }
__device__ __forceinline__ bool operator<=(df64 a, df64 b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(df64 a, df64 b) { return !(a < b); }

__device__ __forceinline__ bool operator!=(df64 a, df64 b) { return a.hi != b.hi || a.lo != b.lo; }

__device__ __forceinline__ df64 fabs(df64 a) { return a.hi < 0.f ? -a : a; }
__device__ __forceinline__ df64 copysign(df64 a, df64 s) { return (a.hi < 0.f) != (s.hi < 0.f) ? -a : a; }

// sqrt by one Newton correction of the float root: x + (a - x^2) / (2x)
__device__ __forceinline__ df64 sqrt(df64 a) {
  if (!(a.hi > 0.f)) return df64(0.f);
  const float x = sqrtf(a.hi);
  const df64 r = a - two_prod(x, x);
  return fast_two_sum(x, __fdiv_rn(r.hi, __fmul_rn(2.f, x)));
}

// ---------------------------------------------------------------- fused double-float expressions
// Sums of products renormalised once: the high parts of the products exactly
// (TwoProd), the high parts summed by TwoSum, every low-order term (the
// products' cross terms and the TwoSum errors) summed in float, one final
// Fast-TwoSum.  Same error class as the operation-by-operation forms (about
// 2^-47 of the largest term), fewer instructions.

// a b + c d
__device__ __forceinline__ df64 dot2(df64 a, df64 b, df64 c, df64 d) {
  const df64 p = two_prod(a.hi, b.hi), q = two_prod(c.hi, d.hi);
  const df64 s = two_sum(p.hi, q.hi);
  float lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  lo = __fmaf_rn(c.hi, d.lo, __fmaf_rn(c.lo, d.hi, __fadd_rn(lo, q.lo)));
  return fast_two_sum(s.hi, __fadd_rn(s.lo, lo));
}

// m - a b - c d
__device__ __forceinline__ df64 fms2(df64 m, df64 a, df64 b, df64 c, df64 d) {
  const df64 p = two_prod(a.hi, b.hi), q = two_prod(c.hi, d.hi);
  const df64 s1 = two_sum(m.hi, -p.hi);
  const df64 s2 = two_sum(s1.hi, -q.hi);
  float lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  lo = __fmaf_rn(c.hi, d.lo, __fmaf_rn(c.lo, d.hi, __fadd_rn(lo, q.lo)));
  const float t = __fadd_rn(__fadd_rn(m.lo, s1.lo), __fsub_rn(s2.lo, lo));
  return fast_two_sum(s2.hi, t);
}

// m - a b
__device__ __forceinline__ df64 fms1(df64 m, df64 a, df64 b) {
  const df64 p = two_prod(a.hi, b.hi);
  const df64 s = two_sum(m.hi, -p.hi);
  const float lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return fast_two_sum(s.hi, __fsub_rn(__fadd_rn(m.lo, s.lo), lo));
}

// y + a x + b w for float a, b
__device__ __forceinline__ df64 fma2_df(float a, df64 x, float b, df64 w, df64 y) {
  const df64 p = two_prod(a, x.hi), q = two_prod(b, w.hi);
  const df64 s1 = two_sum(y.hi, p.hi);
  const df64 s2 = two_sum(s1.hi, q.hi);
  const float lo = __fmaf_rn(a, x.lo, __fmaf_rn(b, w.lo, __fadd_rn(p.lo, q.lo)));
  return fast_two_sum(s2.hi, __fadd_rn(__fadd_rn(y.lo, s1.lo), __fadd_rn(s2.lo, lo)));
}

// y + a x + b w + c v for float a, b, c
__device__ __forceinline__ df64 fma3_df(float a, df64 x, float b, df64 w, float c, df64 v, df64 y) {
  const df64 p = two_prod(a, x.hi), q = two_prod(b, w.hi), r = two_prod(c, v.hi);
  const df64 s1 = two_sum(y.hi, p.hi);
  const df64 s2 = two_sum(s1.hi, q.hi);
  const df64 s3 = two_sum(s2.hi, r.hi);
  const float lo = __fmaf_rn(a, x.lo, __fmaf_rn(b, w.lo, __fmaf_rn(c, v.lo, __fadd_rn(__fadd_rn(p.lo, q.lo), r.lo))));
  const float t = __fadd_rn(__fadd_rn(__fadd_rn(y.lo, s1.lo), __fadd_rn(s2.lo, s3.lo)), lo);
  return fast_two_sum(s3.hi, t);
}

// The same three sums without the final renormalisation (an intermediate
// that only feeds exact products: its low part may exceed half an ulp)
__device__ __forceinline__ df64 fma_df_nr(float a, df64 x, df64 y) {
  df64 p = two_prod(a, x.hi);
  p.lo = __fmaf_rn(a, x.lo, p.lo);
  const df64 s = two_sum(p.hi, y.hi);
  return df64(s.hi, __fadd_rn(s.lo, __fadd_rn(p.lo, y.lo)));
}
__device__ __forceinline__ df64 fma2_df_nr(float a, df64 x, float b, df64 w, df64 y) {
  const df64 p = two_prod(a, x.hi), q = two_prod(b, w.hi);
  const df64 s1 = two_sum(y.hi, p.hi);
  const df64 s2 = two_sum(s1.hi, q.hi);
  const float lo = __fmaf_rn(a, x.lo, __fmaf_rn(b, w.lo, __fadd_rn(p.lo, q.lo)));
  return df64(s2.hi, __fadd_rn(__fadd_rn(y.lo, s1.lo), __fadd_rn(s2.lo, lo)));
}
__device__ __forceinline__ df64 fma3_df_nr(float a, df64 x, float b, df64 w, float c, df64 v, df64 y) {
  const df64 p = two_prod(a, x.hi), q = two_prod(b, w.hi), r = two_prod(c, v.hi);
  const df64 s1 = two_sum(y.hi, p.hi);
  const df64 s2 = two_sum(s1.hi, q.hi);
  const df64 s3 = two_sum(s2.hi, r.hi);
  const float lo = __fmaf_rn(a, x.lo, __fmaf_rn(b, w.lo, __fmaf_rn(c, v.lo, __fadd_rn(__fadd_rn(p.lo, q.lo), r.lo))));
  return df64(s3.hi, __fadd_rn(__fadd_rn(__fadd_rn(y.lo, s1.lo), __fadd_rn(s2.lo, s3.lo)), lo));
}

// ---------------------------------------------------------------- conversions used by the kernels
__device__ __forceinline__ float to_float(float a) { return a; }
__device__ __forceinline__ float to_float(double a) { return narrow(a); }
__device__ __forceinline__ float to_float(df64 a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ double to_double(float a) { return widen(a); }
__device__ __forceinline__ double to_double(double a) { return a; }
__device__ __forceinline__ double to_double(df64 a) { return widen(a.hi) + widen(a.lo); }

// A float or double value in the type T of a state, covariance or
// transport variable (float, double or double-float).
template <class T> struct FromF;
template <> struct FromF<float> {
  __device__ static float get(float a) { return a; }
  __device__ static float get(double a) { return narrow(a); }
};
template <> struct FromF<double> {
  __device__ static double get(float a) { return widen(a); }
  __device__ static double get(double a) { return a; }
};

template <class E> struct ToE;
template <> struct ToE<float> {
  template <class T> __device__ static float get(T a) { return to_float(a); }
};
template <> struct ToE<double> {
  template <class T> __device__ static double get(T a) { return to_double(a); }
};
struct df64;
template <> struct ToE<df64> {
  __device__ static df64 get(df64 a) { return a; }
  __device__ static df64 get(double a) { return df64(a); }
  __device__ static df64 get(float a) { return df64(a); }
};
template <class E, class T> __device__ __forceinline__ E to_e(T a) { return ToE<E>::get(a); }
template <> struct FromF<df64> {
  __device__ static df64 get(float a) { return df64(a); }
  __device__ static df64 get(double a) { return df64(a); }
};
template <class T, class V> __device__ __forceinline__ T conv(V a) { return FromF<T>::get(a); }

// (c - p) converted to E, with c a float cluster coordinate and p a state entry
__device__ __forceinline__ float diff_f(float c, float p) { return c - p; }
__device__ __forceinline__ float diff_f(float c, double p) { return narrow(widen(c) - p); }
__device__ __forceinline__ float diff_f(float c, df64 p) { return to_float(df64(c) - p); }
template <class E, class S> struct DiffTo {
  __device__ static E get(float c, S p) { return (E)diff_f(c, p); }
};
template <class S> struct DiffTo<double, S> {
  __device__ static double get(float c, S p) { return widen(c) - to_double(p); }
};
template <class E, class S> __device__ __forceinline__ E diff_to(float c, S p) { return DiffTo<E, S>::get(c, p); }

// |a| > b, evaluated in the precision of a (the threshold comes in that precision)
__device__ __forceinline__ bool abs_exceeds(float a, float b) { return fabsf(a) > b; }
__device__ __forceinline__ bool abs_exceeds(double a, double b) { return fabs(a) > b; }
__device__ __forceinline__ bool abs_exceeds(df64 a, float b) { return fabsf(to_float(a)) > b; }

// |a| < b (false for NaN), evaluated in the precision of a
__device__ __forceinline__ bool abs_below(float a, float b) { return fabsf(a) < b; }
__device__ __forceinline__ bool abs_below(double a, double b) { return fabs(a) < b; }
__device__ __forceinline__ bool abs_below(df64 a, float b) { return fabsf(to_float(a)) < b; }

template <class T> struct is_df64 { static constexpr bool value = false; };
template <> struct is_df64<df64> { static constexpr bool value = true; };

}  // namespace tpct
