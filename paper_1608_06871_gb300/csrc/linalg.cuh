// Batched dense linear algebra on the GPU (row-major, FP64 real or complex).
//
// These are the dense building blocks of the direct solver of Sec. 2: the leaf
// factorisations, the interface systems of the merges and the exterior
// coupling system are LU factorisations with partial pivoting; every other
// step is a (batched) matrix product.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace hs {

enum { OP_N = 0, OP_T = 1 };

// C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b] for b < batch, row-major,
// op = identity or plain transpose (no conjugation).  beta == 0 never reads C.
template <typename TA, typename TB, typename TC>
void gemm(cudaStream_t s, int opA, int opB, int m, int n, int k, TC alpha, const TA* A, int lda,
          long long sA, const TB* B, int ldb, long long sB, TC beta, TC* C, int ldc, long long sC,
          int batch);

// In-place LU with partial pivoting P A = L U of a batch of n x n matrices.
// piv[j] (0-based) is the row swapped with row j at step j.  info[b] is set to
// j+1 at the first exactly-zero pivot of matrix b (it must be zeroed first).
template <typename E>
void lu_factor(cudaStream_t s, E* A, int lda, long long sA, int n, int* piv, long long sP, int* info,
               int batch);

// Inv[b] = A[b]^{-1} (n x n, leading dimension ldi) from the factors of
// lu_factor (identity right-hand sides through lu_solve).
template <typename E>
void lu_inverse(cudaStream_t s, const E* A, int lda, long long sA, int n, const int* piv, long long sP, E* Inv,
                int ldi, long long sI, int batch);

// Factor the panel columns [j0, j0 + nb) (nb <= 32) of the batch with row
// pivoting and apply the row swaps to whole rows (panel.cu); piv[j0 .. j0+nb)
// receives the swaps, piv[j0+nb .. n) is used as scratch.
template <typename E>
void lu_panel(cudaStream_t s, E* A, int lda, long long sA, int n, int j0, int nb, int* piv, long long sP, int* info,
              int batch);

// Solve A X = B (trans = OP_N) or A^T X = B (trans = OP_T) in place in B
// (n x nrhs, leading dimension ldb) from the factors of lu_factor.
template <typename E>
void lu_solve(cudaStream_t s, int trans, const E* A, int lda, long long sA, int n, const int* piv,
              long long sP, E* B, int ldb, long long sB, int nrhs, int batch);


// FP32 products on the tensor cores by a two-term TF32 split (tc32.cu):
// C = alpha A B + beta C, row-major, no transposes; mode 2: complex A and B,
// mode 1: real A, complex B, mode 0: real A and B (alpha, beta real: .x).
// Leading dimensions and batch strides of A and B in floats, of C in
// elements.  Returns false (nothing launched) when the product cannot run
// there (switched off, or no scratch while the stream is being captured).
bool t32_gemm(cudaStream_t s, int mode, int m, int n, int k, float2 alpha, const float* A, long long lda,
              long long sA, const float* B, long long ldb, long long sB, float2 beta, void* C, int ldc, long long sC,
              int batch);
bool t32_timed_out(cudaStream_t s);
// gemm() measures, once per shape, the tensor-core and the SIMT product and
// keeps the faster (g_autotune; off: a fixed size rule); g_last_gemm_tc is 1
// when the calling thread's last gemm() ran on the tensor cores.
extern bool g_autotune;
extern float g_tc_margin;  // the tensor cores are kept where they take < g_tc_margin of the SIMT time

// Tensor-core use for FP32 products (hs_set_tensor_cores): 0 never; 1 (the
// default) where the per-shape measurement finds them clearly faster; 2 every
// supported product.
extern int g_t32_mode;
extern thread_local bool g_prof_suspended;
extern thread_local int g_last_gemm_tc;
// Synchronises s, then reads and clears this device's flags that a bounded
// tensor-core wait gave up (the split-TF32 product's, the emulated-FP64 one's,
// and the one the host raises in tests; tcgemm.cu).
bool tc_timed_out(cudaStream_t s);
bool oz_timed_out(cudaStream_t s);
cudaError_t tc_raise_timeout_flag();

// FP64 products on the tensor cores by exact BF16 slices (ozaki.cu).  A strided
// FP64 view: element (b, i, k) at p[b sb + (i / ig) si + (i % ig) sg + k sk]
// (ig = 2 reads the real and imaginary parts of complex rows as two real rows).
struct OzView {
  double* p;
  long long sb, si, sg, sk;
  int ig;
};
extern bool g_oz_enabled;
// Scratch bytes of ozaki_gemm for these sizes.
size_t ozaki_scratch_bytes(int m, int n, int k, int batch, bool b_shared);
// C[b] = alpha A[b] B[b] + beta C[b] (m x n, k inner; beta = 0 never reads C)
// with A given row-wise (A(b, i, kk)) and B by its transpose Bt(b, j, kk);
// b_shared: one B for every batch.  Returns cudaErrorNotSupported when the
// tensor-map encoder is unavailable, cudaErrorInvalidValue on bad sizes.
cudaError_t ozaki_gemm(cudaStream_t s, int m, int n, int k, int batch, double alpha, OzView A, OzView Bt,
                       bool b_shared, double beta, OzView C, void* scratch, size_t scratch_bytes);
// The same in two steps, for an operand used by many products: oz_slice cuts
// the rows of a view (A's rows with is_a, or B's columns through Bt) into
// oz_operand_bytes of slices, once; oz_multiply multiplies two sliced operands.
size_t oz_operand_bytes(int rows, int k, int batch, bool is_a);
void oz_slice(cudaStream_t s, OzView v, int rows, int k, int batch, bool is_a, void* buf);
cudaError_t oz_multiply(cudaStream_t s, int m, int n, int k, int batch, double alpha, const void* Aop, const void* Bop,
                        bool b_shared, double beta, OzView C);
// Split-k form for products with few output tiles and a long k: an operand
// sliced "wide" (every piece of k side by side in one row, oz_wide_bytes) is
// multiplied by one launch with the pieces along grid.z into per-piece FP64
// planes (oz_partial_bytes), which oz_zmul_wide sums in order for a complex
// product C (m x n, ldc) = alpha A B + beta C from the real and imaginary
// parts of A (rows) and of B^T (rows); partials: 4 oz_partial_bytes.
size_t oz_wide_bytes(int rows, int k, bool is_a);
size_t oz_partial_bytes(int m, int n, int k);
void oz_slice_wide(cudaStream_t s, OzView v, int rows, int k, bool is_a, void* buf);
cudaError_t oz_multiply_wide(cudaStream_t s, int m, int n, int k, const void* Aop, const void* Bop, double* partial);
cudaError_t oz_zmul_wide(cudaStream_t s, int m, int n, int k, const void* Are, const void* Aim, const void* Bre,
                         const void* Bim, double alpha, double beta, double2* C, int ldc, void* partials);
// The left operand of the Jacobian's x-projection for the pairs c0 .. c0 + nc - 1
// of d * P + p, sliced straight from the fields: rows 2 (c nX + gy) + part of
// u_d z_p over gx (2 nc nX rows, k = nX; oz_operand_bytes(2 nc nX, nX, 1, true)).
void oz_slice_khatri_rao(cudaStream_t s, const double2* Ug, const double2* Zg, int P, int nX, long long c0, int nc,
                         void* buf);

}  // namespace hs
