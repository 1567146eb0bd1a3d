// Helix transport in x and Kalman-filter arithmetic shared by the tracklet
// and refit kernels of the CUDA path.
//
// State p = (y, z, sin phi, tan lambda, q/pT) at a pad-row x; covariance in
// packed lower-triangular order 00,10,11,20,21,22,30,31,32,33,40,41,42,43,44.
#pragma once
#include <type_traits>
#include "tpct_internal.cuh"

namespace tpct {

// g(h) = asin(h)/h and g'(h).  Near 0 from the Taylor series of asin
// (coefficients a_n = (2n)! / (4^n (n!)^2 (2n+1))); float uses it up to
// |h| = 0.25, double up to |h| = 0.01 (truncation below 1e-9 and 1e-25).
template <class E>
__device__ __forceinline__ void asin_ratio(E h, E& g, E& gp) {
  const E u = h * h;
  const E lim = sizeof(E) == 4 ? (E)0.0625 : (E)1e-4;
  if (u < lim) {
    g = (E)1 + u * ((E)(1.0 / 6.0) + u * ((E)(3.0 / 40.0) + u * ((E)(5.0 / 112.0) +
        u * ((E)(35.0 / 1152.0) + u * (E)(63.0 / 2816.0)))));
    gp = h * ((E)(1.0 / 3.0) + u * ((E)(3.0 / 10.0) + u * ((E)(15.0 / 56.0) +
         u * ((E)(35.0 / 144.0) + u * (E)(315.0 / 1408.0)))));
  } else {
    const E ih = (E)1 / h;
    g = asin(h) * ih;
    gp = ((E)1 / sqrt((E)1 - u) - g) * ih;
  }
}

// Double-float version: the series to u^11 below |h| = 0.25 (truncation
// ~2e-17; 4 terms suffice below |h| = 0.01), else g, g' from double asin.
// a_n = binom(2n, n) / (4^n (2n + 1)) as double-float pairs: series of g and of g'/h
constexpr int kAsinTerms = 12;
__constant__ float kAsinG[kAsinTerms][2] = {
#define TPCT_DF(v) {(float)(v), (float)((v) - (double)(float)(v))}
    TPCT_DF(1.0), TPCT_DF(1.0 / 6.0), TPCT_DF(3.0 / 40.0), TPCT_DF(5.0 / 112.0), TPCT_DF(35.0 / 1152.0),
    TPCT_DF(63.0 / 2816.0), TPCT_DF(231.0 / 13312.0), TPCT_DF(143.0 / 10240.0), TPCT_DF(6435.0 / 557056.0),
    TPCT_DF(12155.0 / 1245184.0), TPCT_DF(46189.0 / 5505024.0), TPCT_DF(88179.0 / 12058624.0)};
__constant__ float kAsinD[kAsinTerms][2] = {
    TPCT_DF(0.0), TPCT_DF(2.0 / 6.0), TPCT_DF(12.0 / 40.0), TPCT_DF(30.0 / 112.0), TPCT_DF(280.0 / 1152.0),
    TPCT_DF(630.0 / 2816.0), TPCT_DF(2772.0 / 13312.0), TPCT_DF(2002.0 / 10240.0), TPCT_DF(102960.0 / 557056.0),
    TPCT_DF(218790.0 / 1245184.0), TPCT_DF(923780.0 / 5505024.0), TPCT_DF(1939938.0 / 12058624.0)};
#undef TPCT_DF

__device__ __forceinline__ void asin_ratio(df64 h, df64& g, df64& gp) {
  const df64 u = h * h;
  if (u.hi < 0.0625f) {
    const int top = u.hi < 1e-4f ? 4 : kAsinTerms - 1;
    df64 sg(kAsinG[top][0], kAsinG[top][1]), sd(kAsinD[top][0], kAsinD[top][1]);
    for (int n = top - 1; n >= 1; --n) {
      sg = sg * u + df64(kAsinG[n][0], kAsinG[n][1]);
      sd = sd * u + df64(kAsinD[n][0], kAsinD[n][1]);
    }
    g = sg * u + df64(1.0f);
    gp = h * sd;
  } else {
    const double hd = to_double(h);
    const double gd = asin(hd) / hd;
    g = df64(gd);
    gp = df64((1.0 / sqrt(1.0 - hd * hd) - gd) / hd);
  }
}

// Increments and Jacobian of one exact helix step of length dx in x.
template <class E>
struct Step {
  E dy, dz, ds;                 // increments of y, z, sin phi
  E j_ys, j_yq;                 // d y1 / d sin phi0, d y1 / d q/pT
  E j_zs, j_zt, j_zq;           // d z1 / d sin phi0, d tan l, d q/pT
  E j_sq;                       // d sin phi1 / d q/pT
};

// s1 = s0 + rho dx with rho = -kb q/pT; the chord has the slope of the mean
// direction, (s0 + s1) / (c0 + c1); its signed length L (sign of dx) spans
// an arc L g(rho L / 2); z advances by tan(lambda) times the arc.
template <class E> __device__ __forceinline__ E rsqrt_of(E v) { return rsqrt(v); }
template <> __device__ __forceinline__ float rsqrt_of<float>(float v) { return rsqrtf(v); }
__device__ __forceinline__ df64 rsqrt_of(df64 v) { return df64(1.0f) / sqrt(v); }

template <class E>
__device__ __forceinline__ bool helix_step(E s0, E tl, E qpt, E dx, E kb, E smax, Step<E>& st) {
  const E rho = -kb * qpt;
  const E ds = rho * dx;
  const E s1 = s0 + ds;
  if (!(fabs(s0) < smax && fabs(s1) < smax)) return false;
  // cos phi and tan phi from reciprocal square roots (no divisions)
  const E u0 = (E)1 - s0 * s0, u1 = (E)1 - s1 * s1;
  const E ir0 = rsqrt_of(u0), ir1 = rsqrt_of(u1);
  const E c0 = u0 * ir0, c1 = u1 * ir1;
  const E q0 = s0 * ir0, q1 = s1 * ir1;
  const E ib = (E)1 / (c0 + c1);
  const E slope = (s0 + s1) * ib;
  const E dy = dx * slope;
  const E l2 = dx * dx + dy * dy;
  const E il = l2 > (E)0 ? rsqrt_of(l2) : (E)0;
  const E len = copysign(l2 * il, dx);
  const E h = (E)0.5 * rho * len;
  E g, gp;
  asin_ratio(h, g, gp);
  const E arc = len * g;
  st.dy = dy;
  st.dz = tl * arc;
  st.ds = ds;
  st.j_ys = dx * ((E)2 + slope * (q0 + q1)) * ib;
  st.j_yq = -kb * dx * dx * ((E)1 + slope * q1) * ib;
  // dL/d(dy) = dy / L with the signed L, i.e. sign(dx) * dy / |L|
  const E dy_l = dy * il;
  const E darc_ddy = (g + h * gp) * (dx < (E)0 ? -dy_l : dy_l);
  st.j_zs = tl * darc_ddy * st.j_ys;
  st.j_zq = tl * (darc_ddy * st.j_yq - kb * (E)0.5 * len * len * gp);
  st.j_zt = arc;
  st.j_sq = -kb * dx;
  return true;
}

// C <- F C F^T for F = I + a e02 + b e04 + c e12 + d e13 + e e14 + f e24.
template <class C, class J>
__device__ __forceinline__ void cov_transport(C* m, J a, J b, J c, J d, J e, J f) {
  const C m00 = m[0], m10 = m[1], m11 = m[2], m20 = m[3], m21 = m[4], m22 = m[5];
  const C m30 = m[6], m31 = m[7], m32 = m[8], m33 = m[9];
  const C m40 = m[10], m41 = m[11], m42 = m[12], m43 = m[13], m44 = m[14];
  // rows of G = F C that differ from C
  const C g00 = m00 + a * m20 + b * m40, g02 = m20 + a * m22 + b * m42, g04 = m40 + a * m42 + b * m44;
  const C g10 = m10 + c * m20 + d * m30 + e * m40, g11 = m11 + c * m21 + d * m31 + e * m41;
  const C g12 = m21 + c * m22 + d * m32 + e * m42, g13 = m31 + c * m32 + d * m33 + e * m43;
  const C g14 = m41 + c * m42 + d * m43 + e * m44;
  const C g20 = m20 + f * m40, g21 = m21 + f * m41, g22 = m22 + f * m42;
  const C g23 = m32 + f * m43, g24 = m42 + f * m44;
  // G F^T, lower triangle
  m[0] = g00 + a * g02 + b * g04;
  m[1] = g10 + a * g12 + b * g14;
  m[2] = g11 + c * g12 + d * g13 + e * g14;
  m[3] = g20 + a * g22 + b * g24;
  m[4] = g21 + c * g22 + d * g23 + e * g24;
  m[5] = g22 + f * g24;
  m[6] = m30 + a * m32 + b * m43;
  m[7] = m31 + c * m32 + d * m33 + e * m43;
  m[8] = m32 + f * m43;
  m[10] = m40 + a * m42 + b * m44;
  m[11] = m41 + c * m42 + d * m43 + e * m44;
  m[12] = m42 + f * m44;
}

// Double-float covariance with float Jacobian entries: the same products,
// the two or three terms of each entry summed with one renormalisation (the
// rows of F C, which only feed the exact products of the second stage, are
// left unrenormalised).
__device__ __forceinline__ void cov_transport(df64* m, float a, float b, float c, float d, float e, float f) {
  const df64 m00 = m[0], m10 = m[1], m11 = m[2], m20 = m[3], m21 = m[4], m22 = m[5];
  const df64 m30 = m[6], m31 = m[7], m32 = m[8], m33 = m[9];
  const df64 m40 = m[10], m41 = m[11], m42 = m[12], m43 = m[13], m44 = m[14];
  const df64 g00 = fma2_df_nr(a, m20, b, m40, m00);
  const df64 g02 = fma2_df_nr(a, m22, b, m42, m20);
  const df64 g04 = fma2_df_nr(a, m42, b, m44, m40);
  const df64 g10 = fma3_df_nr(c, m20, d, m30, e, m40, m10);
  const df64 g11 = fma3_df_nr(c, m21, d, m31, e, m41, m11);
  const df64 g12 = fma3_df_nr(c, m22, d, m32, e, m42, m21);
  const df64 g13 = fma3_df_nr(c, m32, d, m33, e, m43, m31);
  const df64 g14 = fma3_df_nr(c, m42, d, m43, e, m44, m41);
  const df64 g20 = fma_df_nr(f, m40, m20), g21 = fma_df_nr(f, m41, m21), g22 = fma_df_nr(f, m42, m22);
  const df64 g23 = fma_df_nr(f, m43, m32), g24 = fma_df_nr(f, m44, m42);
  m[0] = fma2_df(a, g02, b, g04, g00);
  m[1] = fma2_df(a, g12, b, g14, g10);
  m[2] = fma3_df(c, g12, d, g13, e, g14, g11);
  m[3] = fma2_df(a, g22, b, g24, g20);
  m[4] = fma3_df(c, g22, d, g23, e, g24, g21);
  m[5] = fma_df(f, g24, g22);
  m[6] = fma2_df(a, m32, b, m43, m30);
  m[7] = fma3_df(c, m32, d, m33, e, m43, m31);
  m[8] = fma_df(f, m43, m32);
  m[10] = fma2_df(a, m42, b, m44, m40);
  m[11] = fma3_df(c, m42, d, m43, e, m44, m41);
  m[12] = fma_df(f, m44, m42);
}

// Jacobian entries enter as C, except for double-float C where the float
// entries multiply directly (the fused overload above).
template <class C, class E>
__device__ __forceinline__ void cov_transport(C* m, const Step<E>& st) {
  using J = typename std::conditional<is_df64<C>::value, E, C>::type;
  cov_transport(m, conv<J>(st.j_ys), conv<J>(st.j_yq), conv<J>(st.j_zs), conv<J>(st.j_zt), conv<J>(st.j_zq),
                conv<J>(st.j_sq));
}

// chi2 of residual (r0, r1) against S = C[yz] + diag(vy, vz)
template <class C>
__device__ __forceinline__ C kf_chi2(const C* m, C r0, C r1, C vy, C vz) {
  const C s00 = m[0] + vy, s01 = m[1], s11 = m[2] + vz;
  return (r0 * (s11 * r0 - s01 * r1) + r1 * (s00 * r1 - s01 * r0)) / (s00 * s11 - s01 * s01);
}

// a b + c d and m - a b - c d: for float and double the plain expressions (as
// the compiler contracts them); double-float has fused overloads (df64.cuh)
// that renormalise once per expression.
template <class T> __device__ __forceinline__ T dot2(T a, T b, T c, T d) { return a * b + c * d; }
template <class T> __device__ __forceinline__ T fms2(T m, T a, T b, T c, T d) { return (m - a * b) - c * d; }

// Gain K = C H^T S^-1; p += K r; C -= K H C (lower triangle).  Each entry
// of C takes its two gain terms one after the other, which contracts into
// two fused multiply-adds (instead of a product, a multiply-add and a
// subtraction): 30 FP64 operations for the 15 entries.
template <class C, class S>
__device__ __forceinline__ void kf_update_inv(S* p, C* m, C r0, C r1, C s00, C s01, C s11, C idet) {
  const C i00 = s11 * idet, i01 = -s01 * idet, i11 = s00 * idet;
  const C c0[5] = {m[0], m[1], m[3], m[6], m[10]};
  const C c1[5] = {m[1], m[2], m[4], m[7], m[11]};
  C k0[5], k1[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    k0[i] = dot2(c0[i], i00, c1[i], i01);
    k1[i] = dot2(c0[i], i01, c1[i], i11);
    p[i] += (S)(k0[i] * r0 + k1[i] * r1);
  }
  int idx = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j, ++idx) m[idx] = fms2(m[idx], k0[i], c0[j], k1[i], c1[j]);
}

template <class C, class S>
__device__ __forceinline__ void kf_update(S* p, C* m, C r0, C r1, C vy, C vz) {
  const C s00 = m[0] + vy, s01 = m[1], s11 = m[2] + vz;
  kf_update_inv<C, S>(p, m, r0, r1, s00, s01, s11, (C)1 / (s00 * s11 - s01 * s01));
}

// Update that also returns the chi2 of the residual (one reciprocal).
template <class C, class S>
__device__ __forceinline__ C kf_chi2_update(S* p, C* m, C r0, C r1, C v) {
  const C s00 = m[0] + v, s01 = m[1], s11 = m[2] + v;
  const C idet = (C)1 / (s00 * s11 - s01 * s01);
  const C chi2 = (r0 * (s11 * r0 - s01 * r1) + r1 * (s00 * r1 - s01 * r0)) * idet;
  kf_update_inv<C, S>(p, m, r0, r1, s00, s01, s11, idet);
  return chi2;
}

// chi2 test and, if it passes, the update, sharing one reciprocal.
template <class C, class S>
__device__ __forceinline__ bool kf_test_update(S* p, C* m, C r0, C r1, C v, C chi2_max) {
  const C s00 = m[0] + v, s01 = m[1], s11 = m[2] + v;
  const C idet = (C)1 / (s00 * s11 - s01 * s01);
  const C chi2 = (r0 * (s11 * r0 - s01 * r1) + r1 * (s00 * r1 - s01 * r0)) * idet;
  if (!(chi2 <= chi2_max)) return false;
  kf_update_inv<C, S>(p, m, r0, r1, s00, s01, s11, idet);
  return true;
}

// Double-float tracklet filter: the chi2 decision and the state increment
// K r are formed in float (1e-7 relative on a cut decision or on an
// increment much smaller than the state); the gain and the covariance, whose
// update cancels, stay double-float, as two scalar updates (y, then z with
// the residual after the y step; exact for the diagonal cluster covariance).
template <>
__device__ __forceinline__ bool kf_test_update<df64, df64>(df64* p, df64* m, df64 r0, df64 r1, df64 v,
                                                         df64 chi2_max) {
  const df64 s00 = m[0] + v, s01 = m[1], s11 = m[2] + v;
  const float f00 = to_float(s00), f01 = to_float(s01), f11 = to_float(s11);
  const float fr0 = to_float(r0), fr1 = to_float(r1);
  const float chi2 = (fr0 * (f11 * fr0 - f01 * fr1) + fr1 * (f00 * fr1 - f01 * fr0)) / (f00 * f11 - f01 * f01);
  if (!(chi2 <= to_float(chi2_max))) return false;
  const df64 a[5] = {m[0], m[1], m[3], m[6], m[10]};
  const df64 ia = df64(1.0f) / s00;
  df64 k0[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) k0[i] = a[i] * ia;
  int idx = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j, ++idx) m[idx] = fms1(m[idx], k0[i], a[j]);
  const float fr1b = fr1 - to_float(k0[1]) * fr0;
  const df64 b[5] = {m[1], m[2], m[4], m[7], m[11]};
  const df64 ib = df64(1.0f) / (b[1] + v);
  df64 k1[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    k1[i] = b[i] * ib;
    p[i] += df64(to_float(k0[i]) * fr0 + to_float(k1[i]) * fr1b);
  }
  idx = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j, ++idx) m[idx] = fms1(m[idx], k1[i], b[j]);
  return true;
}

// Mixed tracklet filter (double-float state, double covariance, float
// transport and float residuals; S is the state type): the
// chi2 decision in float (1e-6 relative at most, inside the 1e-5 near-cut
// band) and the state increment K r in float (1e-7 of an increment far
// smaller than the state); the gain and the covariance update, whose
// subtraction cancels, in double.
template <class S>
__device__ __forceinline__ bool kf_test_update_mixed(S* p, double* m, float fr0, float fr1, float v,
                                                     float chi2_max) {
  const float f00 = narrow(m[0]) + v, f01 = narrow(m[1]), f11 = narrow(m[2]) + v;
  const float fdet = f00 * f11 - f01 * f01;
  const float chi2 = (fr0 * (f11 * fr0 - f01 * fr1) + fr1 * (f00 * fr1 - f01 * fr0)) / fdet;
  if (!(chi2 <= chi2_max)) return false;
  // The measurement covariance is diagonal (v, v), so the 2-D update is
  // two scalar updates, y then z with the z residual taken after the y step
  // (sequential processing of independent measurements: the same posterior):
  // 25 FP64 operations each instead of 61 for the joint one.  Each 1/S by
  // two Newton-Raphson steps, x <- x + x (1 - S x), from a float seed
  // (about 23 -> 46 -> 53 bits).
  const double vd = widen(v);
  auto recip = [](double s) {
    const float fs = narrow(s);
    double r;
    if (fabsf(fs) > 1e-30f && fabsf(fs) < 1e30f) {
      r = widen(__frcp_rn(fs));
      r = fma(r, fma(-s, r, 1.0), r);
      r = fma(r, fma(-s, r, 1.0), r);
    } else {
      r = 1.0 / s;
    }
    return r;
  };
  // y: column 0 of C
  const double a[5] = {m[0], m[1], m[3], m[6], m[10]};
  const double ia = recip(a[0] + vd);
  double k0[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) k0[i] = a[i] * ia;
  int idx = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j, ++idx) m[idx] = m[idx] - k0[i] * a[j];
  // z: column 1 of the updated C, residual after the y step
  const float fr1b = fr1 - narrow(k0[1]) * fr0;
  const double b[5] = {m[1], m[2], m[4], m[7], m[11]};
  const double ib = recip(b[1] + vd);
  double k1[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    k1[i] = b[i] * ib;
    p[i] += conv<S>(narrow(k0[i]) * fr0 + narrow(k1[i]) * fr1b);
  }
  idx = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j, ++idx) m[idx] = m[idx] - k1[i] * b[j];
  return true;
}

template <class C>
__device__ __forceinline__ void cov_diag(C* m, C vy, C vz, C vs, C vt, C vq) {
#pragma unroll
  for (int i = 0; i < 15; ++i) m[i] = (C)0;
  m[0] = vy; m[2] = vz; m[5] = vs; m[9] = vt; m[14] = vq;
}

}  // namespace tpct
