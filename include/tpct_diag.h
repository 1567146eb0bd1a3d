/*
 * tpct_diag.h -- diagnostics of the GB300 TPC sector tracker library
 * (libtpct.so): instrumentation used by its benchmark and tests, kept apart
 * from the tracking ABI in tpct.h.  None of these has a counterpart in the
 * paper.
 */
#ifndef TPCT_DIAG_H
#define TPCT_DIAG_H

#include "tpct.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Launch count of this context's kernels so far (each kernel launch and each
 * graph kernel node replay counts one). */
int64_t tpct_kernel_launches(const tpct_ctx* ctx);

/* Throughput probe of the FP64 and FP32 FMA pipes: runs `blocks` x 256
 * threads of `iters` independent FMA chains on `stream`, writes nothing to
 * the caller; returns elapsed milliseconds via *ms (synchronises). */
tpct_status tpct_probe_fma(int use_fp64, int blocks, int iters, tpct_stream stream, float* ms);

/* The float <-> double conversions the mixed-precision kernels use instead
 * of the FP64-pipe conversion instructions, applied element-wise on the
 * device: d_out[i] = widen(f_in[i]) and f_out[i] = narrow(d_in[i]) (device
 * arrays of n elements; either pair may be NULL).  widen is exact for zero,
 * normal, infinite and NaN floats and maps float subnormals to zero; narrow
 * rounds to nearest with ties AWAY from zero (the hardware conversion rounds
 * ties to even), flushes results below float's normal range to zero or to a
 * subnormal below 2^-146, saturates beyond float's range to a finite
 * float within 8 ulp of the largest, and turns infinities and NaNs into NaN.  Asynchronous on `stream`. */
tpct_status tpct_diag_convert(const float* f_in, double* d_out, const double* d_in, float* f_out, int64_t n,
                              tpct_stream stream);

#ifdef __cplusplus
}
#endif
#endif
