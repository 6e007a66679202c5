/* at_probe.h -- libat_probe.so: measurement and test helpers beside the
 * solver library (libat_gb300.so, include/at.h).  Not part of the method:
 * the paper has no counterpart.  Plain C ABI, no torch types.
 *
 * Return codes: 0 success, -1 invalid argument, -2 device allocation failed,
 * -3 CUDA error (launch or execution).  Every call is synchronous.
 */
#ifndef AT_PROBE_H
#define AT_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* FP64 FMA throughput of the device: every thread of a full grid runs 8
 * independent fma chains of `iters` steps with `lanes` (1..32) active lanes
 * per warp; best of `reps` launches on `stream` (borrowed, may be NULL).
 * Writes TFLOP/s (2 flops per fma, active lanes only) and the best launch
 * time in ms.  Allocates and frees a small device buffer. */
int at_probe_fp64_fma_lanes(int device, void* stream, int iters, int reps, int lanes, double* tflops,
                            double* ms_best);

/* at_probe_fp64_fma_lanes with all 32 lanes active. */
int at_probe_fp64_fma(int device, void* stream, int iters, int reps, double* tflops, double* ms_best);

/* Latency of one dependent FP64 fma, in SM cycles, with `warps_per_sm`
 * warps per SM each running one dependent chain of `iters` steps. */
int at_probe_fp64_latency(int device, int warps_per_sm, int iters, double* cycles_per_fma);

/* Which pipe an integer operation uses: best-of-`reps` time in ms of a grid
 * (4 CTAs of 256 threads per SM) whose threads run 8 independent chains of
 * `kind` (0 FP64 fma, 1 64-bit integer multiply-add, 2 64-bit integer add,
 * 3 32-bit integer multiply-add) of `iters` steps, beside 8 FP64 fma chains
 * when with_fp64 != 0.  Sharing the FP64 pipe shows as time(kind, 1) close
 * to time(0, 0) + time(kind, 0). */
int at_probe_pipe_mix(int device, int kind, int with_fp64, int iters, int reps, double* ms_best);

/* y[i] = f(x[i]) for device arrays x, y of n doubles (caller-owned device
 * memory, current device): which = 0 the stage kernels' table-driven
 * exponential, 1 CUDA's exp, 2 the stage kernels' Newton reciprocal, 3 IEEE
 * 1/x, 4 the WENO kernels' cubic-step reciprocal.  Runs on the default
 * stream and synchronises the device. */
int at_probe_fn(const double* x, double* y, int64_t n, int which);

#ifdef __cplusplus
}
#endif
#endif
