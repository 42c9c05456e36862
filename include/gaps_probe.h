/* gaps_probe.h -- measurement and test library of the parton-shower library
 * (libgaps_probe.so), kept out of the product library libgaps.so.
 *
 * Nothing here is part of the method: an FP64 throughput probe that the
 * benchmark uses to express the shower's FP64 work in DFMA-equivalents
 * measured on the same device, and builds of numerical building blocks of
 * the kernels (the shower's FP64 logarithm and double -> float conversion,
 * the observables' square root) for the accuracy tests.  Return codes are the
 * gaps_status codes of gaps.h.
 */
#ifndef GAPS_PROBE_H
#define GAPS_PROBE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Measurement helper (no counterpart in the paper): FP64 results per second
 * of this GPU with every SM busy, for DFMA, log, exp, division, sqrt,
 * sincospi and the shower's own logarithm (gaps_log_fp64_*), in
 * host_rates[0..6] (caller-owned, 7 doubles).  device_sink: one device
 * double, never written in practice.  Synchronous; about 60 ms. */
int gaps_probe_fp64_rates(double* device_sink, double* host_rates, void* stream);

/* The FP64 natural logarithm the shower kernels use for the winning trial's
 * scale, ln t' = ln t + ln(r)/c (Eq. (A.5) in log form), and for the dipole
 * cache's ln(z+/z-) (Eq. (A.4)): P. T. P. Tang's table-driven method (ACM
 * TOMS 16 (1990) 378), error below one ulp for positive normal x; other
 * inputs take the CUDA library's log.  y[i] = ln x[i] for 0 <= i < n.
 * _host: host arrays, computed on the calling thread.  _device: device
 * arrays, asynchronous on `stream`.  Both return GAPS_ERR_INVALID for n < 0
 * or a null array with n > 0.  Exported for the accuracy tests. */
int gaps_log_fp64_host(const double* x, double* y, int64_t n);
/* The double -> float conversion (round to nearest even) the kernels do with
 * integer instructions, host build, for the tests: y[i] = (float) x[i].
 * GAPS_ERR_INVALID for n < 0 or a null array with n > 0. */
int gaps_f32_from_f64_host(const double* x, float* y, int64_t n);
int gaps_log_fp64_device(const double* x, double* y, int64_t n, void* stream);
/* The square root the observables kernels take of lengths (|p|, |P|,
 * |p x n_T|, Sec. 3.1 observables): the FP32 reciprocal square root refined
 * by one Newton step in FP64, 1.5e-13 relative for x in 2^-120 .. 2^121;
 * other inputs take the CUDA library's sqrt.  y[i] = sqrt(x[i]) for
 * 0 <= i < n, device arrays, asynchronous on `stream`; GAPS_ERR_INVALID for
 * n < 0 or a null array with n > 0.  Exported for the accuracy tests. */
int gaps_sqrt_obs_device(const double* x, double* y, int64_t n, void* stream);
/* The CUDA error string of the last failed call of this library. */
const char* gaps_probe_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GAPS_PROBE_H */
