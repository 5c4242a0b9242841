/*
 * hs_diag.h -- measurement hooks of libhs (not part of the method; the paper
 * has no counterpart).  Used by the benchmark to time the dominant kernel
 * family inside a timed region and to measure the chip's FP64 arithmetic
 * peak, the denominator of the FP64 roofline.
 *
 * All functions return HS_OK (0) or a negative HS_E* code from hs.h.
 */
#ifndef HS_DIAG_H
#define HS_DIAG_H

#include "hs.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Kernel families that can be timed. */
#define HS_PROF_GEMM_FP64 1 /* the batched FP64 real/complex GEMM kernel */
#define HS_PROF_GEMM_FP32 2 /* the same GEMM kernel in FP32 (mixed-precision path) */

/* Start recording a CUDA event pair around every launch of the given family
 * (on the stream the launch uses) and counting its algorithmic flops
 * (8 m n k per complex product, 4 for real x complex, 2 for real).  Recording
 * is process-wide and not thread-safe.  Errors: HS_EINVAL for an unknown
 * family. */
int hs_prof_start(int family);

/* Stop recording, synchronise on the recorded events and return the summed
 * kernel time in milliseconds, the summed algorithmic flops and the number of
 * launches.  Releases the events.  Any pointer may be NULL. */
int hs_prof_stop(double* total_ms, double* total_flops, long long* launches);

/* Measure the sustained FP64 fused multiply-add rate of `device` with a
 * register-resident kernel of independent DFMA chains on every SM; returns
 * TFLOP/s (2 flops per DFMA) in *tflops.  Runs for about `ms` milliseconds. */
int hs_peak_fp64(int device, double ms, double* tflops);

/* Refinement passes and the last relative change of the far field in the
 * most recent HS_MIXED solve on ctx (0 and -1 before any). */
int hs_refine_stats(const hs_ctx* ctx, int* iterations, double* last_update);

#ifdef __cplusplus
}
#endif
#endif /* HS_DIAG_H */
