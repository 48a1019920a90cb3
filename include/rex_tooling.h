/*
 * rex_tooling.h -- measurement and test tooling of the B300 reweighting library.
 *
 * These entry points are not part of the reweighting ABI (rex.h) and the paper
 * has no counterpart to them.  They live in a separate shared library,
 * librex_tooling_b300.so, built beside librex_b300.so:
 *  - rex_probe_fma measures the FMA issue rate of the device, the denominator of
 *    the exact and mixed kernels' roofline fractions (used by the benchmark);
 *  - rex_probe_convert exposes the integer-ALU float conversions the mixed
 *    kernels use, so that tests can compare them with the hardware conversions.
 *
 * Return value 0 = success, negative = error.  stream is a cudaStream_t passed
 * as void* (NULL = legacy default stream).
 */
#ifndef REX_TOOLING_H
#define REX_TOOLING_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define REX_TOOLING_OK 0
#define REX_TOOLING_EINVAL (-1)   /* null or out-of-range argument */
#define REX_TOOLING_ECUDA (-3)    /* a CUDA call failed */

/* Issue-rate probe of the FP64 (fp64 != 0) or FP32 fused multiply-add pipe of
 * the current device.  Runs a few tens of milliseconds of independent FMA
 * chains on every SM, synchronises stream, and writes the best observed rate in
 * flop/s (an FMA counts two flops).
 * Errors: REX_TOOLING_EINVAL (null output), REX_TOOLING_ECUDA. */
int rex_probe_fma(int fp64, double *flops_per_second, void *stream);

/* The integer-ALU float conversions that the mixed-precision q q~ -> t t~ (g)
 * kernels use in place of FP64-pipe conversions (B300 issues FP64 at 1/64 of
 * the FP32 rate): f32_out[i] = FP64 -> FP32 of in[i] (round to nearest even;
 * magnitudes below 2^-126 give a signed zero, overflow gives infinity, NaN
 * stays NaN), f64_out[i] = FP32 -> FP64 of f32_out[i] (exact) and, if
 * f32_finite_out is not null, f32_finite_out[i] = the kernels' FP64 -> FP32
 * conversion for momenta (the same rounding; finiteness is checked once per
 * event instead, so its value is meaningful for finite in[i] below 2^128 only).
 * Device arrays of n elements; enqueue only.
 * Errors: REX_TOOLING_EINVAL (n < 0, null array), REX_TOOLING_ECUDA. */
int rex_probe_convert(const double *in, int64_t n, float *f32_out, double *f64_out,
                      float *f32_finite_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* REX_TOOLING_H */
