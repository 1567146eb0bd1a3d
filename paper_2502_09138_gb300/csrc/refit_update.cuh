// The Kalman update of the refits (track refit and chain refit): the 2-D
// update of a cluster as two scalar updates, y then z with the z residual
// taken after the y step.  The cluster covariance is diagonal (v, v), so
// this is the joint update's posterior and chi2 (sequential processing of
// independent measurements); it takes one multiply-add per covariance entry
// and scalar step instead of a 2x2 inverse, a 10-entry gain and two
// multiply-adds per entry.
#pragma once

#include "track_math.cuh"

namespace tpct {

// 1/s: double from a float seed and two Newton-Raphson steps (about
// 23 -> 46 -> 53 bits), the other types by their own division
template <class C> __device__ __forceinline__ C refit_recip(C s) { return conv<C>(1.0f) / s; }
template <> __device__ __forceinline__ double refit_recip<double>(double s) {
  const float fs = narrow(s);
  if (!(fabsf(fs) > 1e-30f && fabsf(fs) < 1e30f)) return 1.0 / s;
  double r = widen(__frcp_rn(fs));
  r = fma(r, fma(-s, r, 1.0), r);
  r = fma(r, fma(-s, r, 1.0), r);
  return r;
}

// One scalar step on state component K (0: y, 1: z) with residual res;
// returns its chi2 contribution res^2 / S and, in gz, the step's gain on z.
template <class C, class S, int K>
__device__ __forceinline__ C refit_scalar_step(S* d, C* m, C res, C v, C& gz) {
  constexpr int col[2][5] = {{0, 1, 3, 6, 10}, {1, 2, 4, 7, 11}};   // column K of the lower triangle
  C a[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) a[i] = m[col[K][i]];
  const C is = refit_recip<C>(a[K] + v);
  C g[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    g[i] = a[i] * is;
    d[i] += (S)(g[i] * res);
  }
  int idx = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j, ++idx) m[idx] = m[idx] - g[i] * a[j];
  gz = g[1];
  return res * res * is;
}

// The update with residuals (r0, r1) of (y, z) and cluster variance v in
// both; returns its chi2.
template <class C, class S>
__device__ __forceinline__ C refit_update(S* d, C* m, C r0, C r1, C v) {
  C gz, unused;
  C chi2 = refit_scalar_step<C, S, 0>(d, m, r0, v, gz);
  chi2 += refit_scalar_step<C, S, 1>(d, m, r1 - gz * r0, v, unused);
  return chi2;
}

}  // namespace tpct
