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
#define HS_PROF_GEMM_TC 3   /* the tensor-core complex FP32 GEMM (mixed-precision path) */
#define HS_PROF_GEMM_EMU 4  /* the emulated FP64 product on the tensor cores (FP64-equivalent flops) */

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

/* The same for FP32 fused multiply-adds (independent FFMA chains on every SM):
 * the denominator of the SIMT FP32 GEMM family's roofline. */
int hs_peak_fp32(int device, double ms, double* tflops);

/* Refinement passes, the last relative change of the far field and the
 * estimated relative error of the returned far field (the stopping quantity:
 * the last change times rho / (1 - rho), rho the observed contraction of the
 * passes, or the change itself before rho is known) in the most recent
 * HS_MIXED solve on ctx (0, -1, -1 before any).  Any pointer may be NULL. */
int hs_refine_stats(const hs_ctx* ctx, int* iterations, double* last_update, double* est_error);

/* Device time of the two factorisation phases of the last build on ctx, in
 * milliseconds (CUDA events on the context's stream): the interior (leaf
 * operators and every merge up the tree, Table 1's T_interior) and the
 * exterior (the layer-potential matrices when k is new, the coupled root
 * system and its LU, Table 1's T_bdry).  -1 before any build and after a
 * build replayed from a CUDA graph (HS_MIXED, unchanged k), which is not
 * split.  Any pointer may be NULL. */
int hs_build_phase_ms(const hs_ctx* ctx, double* interior_ms, double* boundary_ms);

/* The same for the adjoint refinement of the most recent HS_MIXED Jacobian,
 * gradient or Gauss-Newton step on ctx: passes, the last relative change of
 * the adjoint fields at the interior nodes and the estimated relative error
 * of the returned ones (0, -1, -1 before any).  Any pointer may be NULL. */
int hs_adjoint_refine_stats(const hs_ctx* ctx, int* iterations, double* last_update, double* est_error);

/* Replay the mixed-precision factorisation from a CUDA graph captured once
 * per frequency (enable != 0, the default) or enqueue it launch by launch
 * (enable == 0).  Process-wide; takes effect at the next hs_build.  The
 * results are bitwise identical either way.  Never fails. */
int hs_set_graphs(int enable);

/* FP32 products (complex x complex, real x complex, real x real; untransposed
 * operands) on the tensor cores by the split-TF32 product: enable == 0 never;
 * 1 (the default) per shape, where measured clearly faster (hs_set_autotune,
 * hs_set_tc_margin); 2 every such product.  Process-wide; takes effect at the
 * next launch.  Errors: HS_EINVAL for other values. */
int hs_set_tensor_cores(int enable);

/* Bytes of scratch the Jacobian contraction may use for one chunk of
 * (incidence, receiver) pairs (their Khatri-Rao rows and half-projected
 * rows); 0 restores the default (1 GiB).  Smaller budgets mean more, smaller
 * chunks with identical results.  Process-wide; takes effect at the next
 * Jacobian.  Never fails. */
int hs_set_contract_budget(unsigned long long bytes);

/* Failure injection for tests of the error paths (host side only; nothing
 * faults, traps or waits on the GPU).
 *
 * hs_fail_next_allocs: the next n device allocations made by any context
 * (its persistent buffers at hs_create or a later first use, or the growth of
 * its per-call workspace) fail without calling cudaMalloc; the call that
 * needed the memory returns HS_ENOMEM with its reason in hs_last_error, and
 * the context stays usable.  n = 0 clears the hook.  Process-wide, not
 * thread-safe.  Errors: HS_EINVAL for n < 0.
 *
 * hs_raise_tc_timeout: sets the tensor-core timeout flag of `device` from the
 * host, exactly as a bounded tensor-core wait that gave up would; the next
 * call on that device that checks the flag (every HS_MIXED build, solve and
 * tensor-core product) returns HS_ETIMEOUT and clears it.  Errors:
 * HS_ECUDA. */
int hs_fail_next_allocs(int n);
int hs_raise_tc_timeout(int device);

/* C[b] = A[b] B[b] for b < batch: complex FP32 (interleaved re, im),
 * row-major, A m x k, B k x n, C m x n, contiguous batches, all DEVICE
 * pointers on the current device, enqueued on `stream` (a cudaStream_t, NULL
 * for the legacy default stream) and synchronised before return.  Uses the
 * library's GEMM dispatch: the tensor-core kernel when hs_set_tensor_cores
 * allows it and the shape is eligible; *used_tc (if not NULL) says which ran.
 * Errors: HS_EINVAL (non-positive size, NULL pointer), HS_ETIMEOUT (a bounded
 * tensor-core wait gave up; C is then unspecified), HS_ECUDA. */
int hs_cgemm32(int m, int n, int k, const void* A, const void* B, void* C, int batch, void* stream,
               int* used_tc);

/* C[b] = A[b] B[b] in FP32 through the library's GEMM dispatch, for the
 * three operand forms of its tensor-core product: mode 2 complex A (m x k) and
 * B (k x n), complex C; mode 1 real A, complex B and C; mode 0 real A, B and C.
 * Row-major, contiguous batches (b_shared != 0: one B for every batch item),
 * DEVICE pointers on the current device, enqueued on `stream` and synchronised
 * before return; *used_tc (if not NULL) is 1 when the tensor cores ran it.
 * Errors: HS_EINVAL (mode outside 0..2, non-positive size, NULL pointer),
 * HS_ETIMEOUT, HS_ECUDA. */
int hs_gemm32(int mode, int m, int n, int k, const void* A, const void* B, void* C, int batch, int b_shared,
              void* stream, int* used_tc);

/* The GEMM dispatch's choice between the tensor-core and the SIMT FP32
 * product: enable != 0 (the default) measures both once per shape, outside
 * stream capture, and keeps the faster; 0 uses a fixed size rule.  Errors:
 * none. */
int hs_set_autotune(int enable);

/* Where the dispatch measures both products, the tensor cores are kept when
 * they take less than `margin` (0 < margin <= 1; default 0.5) of the SIMT
 * product's time.  Applies to shapes measured afterwards.  Errors: HS_EINVAL. */
int hs_set_tc_margin(double margin);

/* C = op(A) op(B) (+ C when accumulate != 0): complex128 (interleaved re,
 * im), row-major, op(A) m x k, op(B) k x n, C m x n; op = transpose when
 * transA / transB != 0 (A stored k x m, B stored n x k), no conjugation.
 * DEVICE pointers on the current device, enqueued on `stream` (a
 * cudaStream_t, NULL for the legacy default stream) and synchronised before
 * return.  Runs the library's FP64 GEMM dispatch (the kernels of the FP64
 * solver and of the mixed path's FP64 refinement).  Errors: HS_EINVAL
 * (non-positive size, NULL pointer), HS_ECUDA. */
int hs_zgemm(int transA, int transB, int m, int n, int k, const void* A, const void* B, void* C, int accumulate,
             void* stream);

/* C[b] = A[b] B[b] for b < batch in FP64 (real, row-major, A m x k, B k x n,
 * C m x n, contiguous batches; DEVICE pointers on the current device,
 * enqueued on `stream` and synchronised before return) by the library's
 * emulated FP64 product on the tensor cores: rows of A and columns of B
 * scaled by powers of two and split into eight exact 7-bit BF16 slices, the
 * 36 slice pairs of weight >= 2^-63 multiplied exactly in FP32 accumulators,
 * recombined exactly in integers and rounded once per piece of at most 384 of
 * k (within the FP64 product's bound 2 k u |A||B|).  Allocates and frees
 * its scratch on `stream`.  Errors: HS_EINVAL (bad size, NULL), HS_ENOMEM,
 * HS_ETIMEOUT (a bounded tensor-core wait gave up), HS_ECUDA (also when the
 * driver offers no tensor-map encoder). */
int hs_dgemm_emulated(int m, int n, int k, const void* A, const void* B, void* C, int batch, void* stream);

/* Use the emulated FP64 product above for the FP64 Jacobian contraction
 * (enable != 0, the default) or the FP64 SIMT GEMM (enable == 0).
 * Process-wide; takes effect at the next Jacobian.  Never fails. */
int hs_set_fp64_emulation(int enable);

/* The two products LSQR applies to the explicit FP32 Jacobian (Sec. 3.3,
 * hs_gn_step_lsqr with products = HS_MIXED): y = J v and g = Re(J^H u) for a
 * complex FP32 J (rows x n, row-major, interleaved re, im), real FP64 v (n),
 * complex FP64 u and y (rows, interleaved) and real FP64 g (n), with FP64
 * products and sums (J's entries widened exactly), so that the two are
 * transposes of one operator to FP64 rounding.  DEVICE pointers on the
 * current device, enqueued on `stream` and synchronised before return;
 * allocates and frees 8 n ceil(rows / 256) bytes of scratch.  Errors:
 * HS_EINVAL (non-positive size, rows > 65535 * 256, NULL pointer),
 * HS_ENOMEM, HS_ECUDA. */
int hs_jacobian32_products(long long rows, int n, const void* J, const double* v, void* y, const void* u, double* g,
                           void* stream);

/* Solve A[b] X[b] = B[b] in place in B for b < batch with the library's
 * batched LU (partial pivoting; tournament pivoting for panels taller than 256
 * rows) and triangular solves: complex (interleaved re, im), row-major,
 * A n x n (overwritten by its factors), B n x nrhs, contiguous batches, DEVICE
 * pointers on the current device, enqueued on `stream` (a cudaStream_t, NULL
 * for the legacy default stream) and synchronised before return.  precision
 * HS_FP64: complex128; HS_MIXED: complex64.  Allocates and frees its pivot
 * and status arrays.  Errors: HS_EINVAL (bad size or precision, NULL
 * pointer), HS_ESINGULAR (an exactly zero pivot), HS_ENOMEM, HS_ECUDA. */
int hs_lu_solve(int precision, int n, int nrhs, void* A, void* B, int batch, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HS_DIAG_H */
