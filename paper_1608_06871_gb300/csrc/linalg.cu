// Batched dense linear algebra kernels (see linalg.cuh).
//
// FP64 on this part runs at a small fraction of the FP32 rate, so these
// kernels are arithmetic-bound by construction; they are tiled for data reuse
// in shared memory and use every SM through the batch and tile dimensions.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include <cooperative_groups.h>

#include "linalg.cuh"

namespace cg = cooperative_groups;

namespace hs {

bool prof_active(int family);
void prof_begin(cudaStream_t s, cudaEvent_t* a);
void prof_end(cudaStream_t s, cudaEvent_t a, double flops);

namespace {
template <typename T> struct is_cplx { static constexpr bool v = false; };
template <> struct is_cplx<double2> { static constexpr bool v = true; };
template <> struct is_cplx<float2> { static constexpr bool v = true; };
template <typename T> struct is_fp64 { static constexpr bool v = false; };
template <> struct is_fp64<double> { static constexpr bool v = true; };
template <> struct is_fp64<double2> { static constexpr bool v = true; };
template <typename TA, typename TB> constexpr double flops_per_mac() {
  return (is_cplx<TA>::v && is_cplx<TB>::v) ? 8.0 : ((is_cplx<TA>::v || is_cplx<TB>::v) ? 4.0 : 2.0);
}
constexpr int BM = 32, BN = 32, BK = 16;  // GEMM tile
constexpr int NB = 32;                    // LU panel / TRSM block size
constexpr int NBB = 128;                  // LU super-panel: k of the trailing updates
constexpr int kMaxCluster = 8;            // portable thread-block cluster size (split-k)

template <typename T> __device__ __forceinline__ T ld_op(const T* P, int ld, int op, int r, int c) {
  return op == OP_N ? P[(long long)r * ld + c] : P[(long long)c * ld + r];
}

// 32 x 32 tile, 2 x 2 outputs per thread.  blockIdx.z = batch * splits + split:
// with splits > 1 the kernel is launched in clusters of `splits` CTAs along z,
// each CTA covers a slice of k, and the partial tiles are summed through
// distributed shared memory in split order (deterministic, no atomics): rank r
// reduces and writes its share of the tile's rows.
template <typename TA, typename TB, typename TC>
__global__ void __launch_bounds__(256) k_gemm(int opA, int opB, int m, int n, int k, TC alpha, const TA* __restrict__ A,
                                              int lda, long long sA, const TB* __restrict__ B, int ldb, long long sB,
                                              TC beta, TC* __restrict__ C, int ldc, long long sC, int splits) {
  constexpr size_t A_BYTES = sizeof(TA) * BK * (BM + 1), B_BYTES = sizeof(TB) * BK * (BN + 1);
  constexpr size_t RED_BYTES = sizeof(TC) * BM * BN;
  __shared__ __align__(16) unsigned char raw[A_BYTES + B_BYTES > RED_BYTES ? A_BYTES + B_BYTES : RED_BYTES];
  TA(*As)[BM + 1] = reinterpret_cast<TA(*)[BM + 1]>(raw);
  TB(*Bs)[BN + 1] = reinterpret_cast<TB(*)[BN + 1]>(raw + A_BYTES);
  const int b = blockIdx.z / splits, sp = blockIdx.z % splits;
  A += b * sA;
  B += b * sB;
  C += b * sC;
  const int kc = ((k + splits - 1) / splits + BK - 1) / BK * BK;
  const int kbeg = sp * kc, kend = min(k, kbeg + kc);
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  TC acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = el<TC>::zero();
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      int r, kk;
      if (opA == OP_N) { r = e / BK; kk = e % BK; } else { kk = e / BM; r = e % BM; }
      int gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < m && gk < kend) ? ld_op(A, lda, opA, gr, gk) : el<TA>::zero();
    }
    for (int e = threadIdx.x; e < BK * BN; e += 256) {
      int kk, c;
      if (opB == OP_N) { kk = e / BN; c = e % BN; } else { c = e / BK; kk = e % BK; }
      int gk = k0 + kk, gc = col0 + c;
      Bs[kk][c] = (gk < kend && gc < n) ? ld_op(B, ldb, opB, gk, gc) : el<TB>::zero();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      TA a0 = As[kk][ty], a1 = As[kk][ty + 16];
      TB b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      acc[0][0] = fmac(acc[0][0], a0, b0);
      acc[0][1] = fmac(acc[0][1], a0, b1);
      acc[1][0] = fmac(acc[1][0], a1, b0);
      acc[1][1] = fmac(acc[1][1], a1, b1);
    }
    __syncthreads();
  }
  if (splits == 1) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
        if (r < m && c < n) {
          TC v = scal<TC, TC>(alpha, acc[i][j]);
          long long o = (long long)r * ldc + c;
          if (!is_zero(beta)) v = addv(v, scal<TC, TC>(beta, C[o]));
          C[o] = v;
        }
      }
    return;
  }
  TC* red = reinterpret_cast<TC*>(raw);  // the k loop ended with a barrier
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) red[(ty + 16 * i) * BN + tx + 16 * j] = acc[i][j];
  cg::cluster_group cl = cg::this_cluster();
  cl.sync();
  const int rows_per = (BM + splits - 1) / splits;
  const int rb = sp * rows_per, re = min(BM, rb + rows_per);
  for (int e = rb * BN + threadIdx.x; e < re * BN; e += 256) {
    TC sum = el<TC>::zero();
    for (int q = 0; q < splits; ++q) sum = addv(sum, cl.map_shared_rank(red, q)[e]);
    const int r = row0 + e / BN, c = col0 + e % BN;
    if (r < m && c < n) {
      TC v = scal<TC, TC>(alpha, sum);
      long long o = (long long)r * ldc + c;
      if (!is_zero(beta)) v = addv(v, scal<TC, TC>(beta, C[o]));
      C[o] = v;
    }
  }
  cl.sync();  // keep this CTA's partial tile alive until every rank has read it
}

// 64 x 64 tile, 4 x 4 outputs per thread (more arithmetic per shared-memory
// load), k-step 8 with the next tile prefetched into registers.  For shapes
// with enough tiles to fill the machine.
constexpr int GB = 64, GK = 8;
// With splits > 1 (8-byte output elements only: the partial tile must fit in
// static shared memory) the kernel runs in clusters of `splits` CTAs along z,
// each over a slice of k, and the partial tiles are summed in split order
// through distributed shared memory, as in k_gemm.
template <typename TA, typename TB, typename TC>
__global__ void __launch_bounds__(256, 2) k_gemm_big(int opA, int opB, int m, int n, int k, TC alpha,
                                                  const TA* __restrict__ A, int lda, long long sA,
                                                  const TB* __restrict__ B, int ldb, long long sB, TC beta,
                                                  TC* __restrict__ C, int ldc, long long sC, int splits) {
  __shared__ TA As[GK][GB];
  __shared__ TB Bs[GK][GB];
  const int b = blockIdx.z / splits, sp = blockIdx.z % splits;
  A += b * sA;
  B += b * sB;
  C += b * sC;
  const int kc = ((k + splits - 1) / splits + GK - 1) / GK * GK;
  const int kbeg = sp * kc, kend = min(k, kbeg + kc);
  const int row0 = blockIdx.y * GB, col0 = blockIdx.x * GB;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  TC acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = el<TC>::zero();
  // each thread stages 2 elements of A and 2 of B per k-step (64 x 8 each)
  TA ra[2];
  TB rb[2];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      int e = threadIdx.x + 256 * q;
      int r, kk;
      if (opA == OP_N) { r = e / GK; kk = e % GK; } else { kk = e / GB; r = e % GB; }
      int gr = row0 + r, gk = k0 + kk;
      ra[q] = (gr < m && gk < kend) ? ld_op(A, lda, opA, gr, gk) : el<TA>::zero();
      int kk2, c;
      if (opB == OP_N) { kk2 = e / GB; c = e % GB; } else { c = e / GK; kk2 = e % GK; }
      int gk2 = k0 + kk2, gc = col0 + c;
      rb[q] = (gk2 < kend && gc < n) ? ld_op(B, ldb, opB, gk2, gc) : el<TB>::zero();
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      int e = threadIdx.x + 256 * q;
      int r, kk;
      if (opA == OP_N) { r = e / GK; kk = e % GK; } else { kk = e / GB; r = e % GB; }
      As[kk][r] = ra[q];
      int kk2, c;
      if (opB == OP_N) { kk2 = e / GB; c = e % GB; } else { c = e / GK; kk2 = e % GK; }
      Bs[kk2][c] = rb[q];
    }
  };
  load(kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += GK) {
    store();
    __syncthreads();
    if (k0 + GK < kend) load(k0 + GK);
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      TA a[4];
      TB bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmac(acc[i][j], a[i], bb[j]);
    }
    __syncthreads();
  }
  if constexpr (sizeof(TC) <= 8) {
    if (splits > 1) {
      __shared__ TC red[GB * GB];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) red[(ty + 16 * i) * GB + tx + 16 * j] = acc[i][j];
      cg::cluster_group cl = cg::this_cluster();
      cl.sync();
      const int rows_per = (GB + splits - 1) / splits;
      const int rb = sp * rows_per, re = min(GB, rb + rows_per);
      for (int e = rb * GB + threadIdx.x; e < re * GB; e += 256) {
        TC sum = el<TC>::zero();
        for (int q = 0; q < splits; ++q) sum = addv(sum, cl.map_shared_rank(red, q)[e]);
        const int r = row0 + e / GB, c = col0 + e % GB;
        if (r < m && c < n) {
          TC v = scal<TC, TC>(alpha, sum);
          long long o = (long long)r * ldc + c;
          if (!is_zero(beta)) v = addv(v, scal<TC, TC>(beta, C[o]));
          C[o] = v;
        }
      }
      cl.sync();  // keep this CTA's partial tile alive until every rank has read it
      return;
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
      if (r < m && c < n) {
        TC v = scal<TC, TC>(alpha, acc[i][j]);
        long long o = (long long)r * ldc + c;
        if (!is_zero(beta)) v = addv(v, scal<TC, TC>(beta, C[o]));
        C[o] = v;
      }
    }
}


// Untransposed FP32 products (real or complex, 4- or 8-byte elements): the
// 64 x 64 tile and 4 x 4 outputs per thread of k_gemm_big, with the operand
// tiles staged by cp.async 16-byte copies into a three-stage shared-memory
// ring (k-step 16), so that the loads of the next two k-steps overlap the
// products of the current one; zero-filled copies cover the edges.  Needs
// 16-byte aligned operand rows (checked by the host).  splits > 1: k split
// over a cluster, partial tiles summed in split order through distributed
// shared memory.
constexpr int PK = 16, PST = 3;
template <typename TA, typename TB, typename TC>
struct PipeCfg {
  static constexpr int A_ST = GB * PK * (int)sizeof(TA);  // bytes of one A stage (64 rows x 16 k)
  static constexpr int B_ST = PK * GB * (int)sizeof(TB);  // bytes of one B stage (16 k x 64 columns)
  static constexpr int RING = PST * (A_ST + B_ST);
  static constexpr int RED = GB * GB * (int)sizeof(TC);
  static constexpr int SMEM = RING > RED ? RING : RED;
};

__device__ __forceinline__ void cp16(void* dst, const void* src, int bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <typename TA, typename TB, typename TC>
__global__ void __launch_bounds__(256, 2) k_gemm_pipe(int m, int n, int k, TC alpha, const TA* __restrict__ A, int lda,
                                                   long long sA, const TB* __restrict__ B, int ldb, long long sB,
                                                   TC beta, TC* __restrict__ C, int ldc, long long sC, int splits) {
  using Cf = PipeCfg<TA, TB, TC>;
  extern __shared__ __align__(16) unsigned char pipe_smem[];
  constexpr int EA = 16 / (int)sizeof(TA), EB = 16 / (int)sizeof(TB);  // elements per 16-byte copy
  const int b = blockIdx.z / splits, sp = blockIdx.z % splits;
  A += b * sA;
  B += b * sB;
  C += b * sC;
  const int kc = ((k + splits - 1) / splits + PK - 1) / PK * PK;
  const int kbeg = sp * kc, kend = min(k, kbeg + kc);
  const int nsteps = kend > kbeg ? (kend - kbeg + PK - 1) / PK : 0;
  const int row0 = blockIdx.y * GB, col0 = blockIdx.x * GB;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  auto As = [&](int st) { return reinterpret_cast<TA*>(pipe_smem + st * (Cf::A_ST + Cf::B_ST)); };
  auto Bs = [&](int st) { return reinterpret_cast<TB*>(pipe_smem + st * (Cf::A_ST + Cf::B_ST) + Cf::A_ST); };
  // stage the k-step `step` into ring slot `st`
  auto issue = [&](int step, int st) {
    const int k0 = kbeg + step * PK;
    TA* as = As(st);
    TB* bs = Bs(st);
    constexpr int CA = GB * PK / EA, CB = PK * GB / EB;  // 16-byte copies per stage
    for (int q = tid; q < CA; q += 256) {
      const int r = q / (PK / EA), kk = (q % (PK / EA)) * EA;
      const int gr = row0 + r, gk = k0 + kk;
      const int valid = (gr < m && gk < kend) ? min(EA, kend - gk) : 0;
      const TA* src = valid ? A + (long long)gr * lda + gk : A;
      cp16(as + r * PK + kk, src, valid * (int)sizeof(TA));
    }
    for (int q = tid; q < CB; q += 256) {
      const int kk = q / (GB / EB), c = (q % (GB / EB)) * EB;
      const int gk = k0 + kk, gc = col0 + c;
      const int valid = (gk < kend && gc < n) ? min(EB, n - gc) : 0;
      const TB* src = valid ? B + (long long)gk * ldb + gc : B;
      cp16(bs + kk * GB + c, src, valid * (int)sizeof(TB));
    }
  };
  TC acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = el<TC>::zero();
#pragma unroll
  for (int st = 0; st < PST - 1; ++st) {
    if (st < nsteps) issue(st, st);
    cp_commit();
  }
  for (int step = 0; step < nsteps; ++step) {
    cp_wait<PST - 2>();
    __syncthreads();  // stage `step` landed for every thread; slot (step - 1) % PST is free
    if (step + PST - 1 < nsteps) issue(step + PST - 1, (step + PST - 1) % PST);
    cp_commit();
    const TA* as = As(step % PST);
    const TB* bs = Bs(step % PST);
#pragma unroll
    for (int kk = 0; kk < PK; ++kk) {
      TA a[4];
      TB bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = as[(ty + 16 * i) * PK + kk];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = bs[kk * GB + tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmac(acc[i][j], a[i], bb[j]);
    }
  }
  cp_wait<0>();
  __syncthreads();
  if (splits > 1) {
    TC* red = reinterpret_cast<TC*>(pipe_smem);  // the ring is free now
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) red[(ty + 16 * i) * GB + tx + 16 * j] = acc[i][j];
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    const int rows_per = (GB + splits - 1) / splits;
    const int rb = sp * rows_per, re = min(GB, rb + rows_per);
    for (int e = rb * GB + tid; e < re * GB; e += 256) {
      TC sum = el<TC>::zero();
      for (int q = 0; q < splits; ++q) sum = addv(sum, cl.map_shared_rank(red, q)[e]);
      const int r = row0 + e / GB, c = col0 + e % GB;
      if (r < m && c < n) {
        TC v = scal<TC, TC>(alpha, sum);
        long long o = (long long)r * ldc + c;
        if (!is_zero(beta)) v = addv(v, scal<TC, TC>(beta, C[o]));
        C[o] = v;
      }
    }
    cl.sync();  // keep this CTA's partial tile alive until every rank has read it
    return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
      if (r < m && c < n) {
        TC v = scal<TC, TC>(alpha, acc[i][j]);
        long long o = (long long)r * ldc + c;
        if (!is_zero(beta)) v = addv(v, scal<TC, TC>(beta, C[o]));
        C[o] = v;
      }
    }
}

__device__ __forceinline__ double shfl(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ float shfl(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double2 shfl(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ float2 shfl(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// Triangular solve with a diagonal block of size nb <= NB for many right-hand
// sides: one warp per right-hand side, lane r holding x_r; each substitution
// step broadcasts the finished unknown with a shuffle.  mode: 0 = L (unit
// lower), 1 = U (upper), 2 = U^T (lower, non-unit), 3 = L^T (upper, unit).
constexpr int TRSM_WARPS = 4;
template <typename E>
__global__ void __launch_bounds__(32 * TRSM_WARPS) k_trsm_diag(const E* A, int lda, long long sA, int i0, int nb,
                                                              int mode, E* B, int ldb, long long sB, int nrhs) {
  __shared__ E T[NB][NB + 1];
  const int b = blockIdx.y;
  A += b * sA;
  B += b * sB;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int r = e / nb, c = e % nb;
    bool tr = (mode >= 2);
    T[r][c] = tr ? A[(long long)(i0 + c) * lda + i0 + r] : A[(long long)(i0 + r) * lda + i0 + c];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.x * TRSM_WARPS + warp;
  if (col >= nrhs) return;  // whole warp leaves together
  E x = lane < nb ? B[(long long)(i0 + lane) * ldb + col] : el<E>::zero();
  const bool lower = (mode == 0 || mode == 2);
  const bool unit = (mode == 0 || mode == 3);
  if (lower) {
    for (int s = 0; s < nb; ++s) {
      if (!unit && lane == s) x = el<E>::div(x, T[s][s]);
      E xs = shfl(x, s);
      if (lane > s && lane < nb) x = fmsc(x, T[lane][s], xs);
    }
  } else {
    for (int s = nb - 1; s >= 0; --s) {
      if (!unit && lane == s) x = el<E>::div(x, T[s][s]);
      E xs = shfl(x, s);
      if (lane < s) x = fmsc(x, T[lane][s], xs);
    }
  }
  if (lane < nb) B[(long long)(i0 + lane) * ldb + col] = x;
}

// Same solve, one thread per right-hand side with the 32 unknowns in
// registers (fully unrolled): the better choice when there are many
// right-hand sides in the batch (leaf and merge systems).
template <typename E>
__global__ void __launch_bounds__(128) k_trsm_diag_col(const E* A, int lda, long long sA, int i0, int nb, int mode,
                                                       E* B, int ldb, long long sB, int nrhs) {
  __shared__ E T[NB][NB + 1];
  const int b = blockIdx.y;
  A += b * sA;
  B += b * sB;
  const bool tr = (mode >= 2);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    int r = e / NB, c = e % NB;
    T[r][c] = (r < nb && c < nb) ? (tr ? A[(long long)(i0 + c) * lda + i0 + r] : A[(long long)(i0 + r) * lda + i0 + c])
                                 : el<E>::zero();
  }
  __syncthreads();
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= nrhs) return;
  E x[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) x[r] = r < nb ? B[(long long)(i0 + r) * ldb + col] : el<E>::zero();
  const bool lower = (mode == 0 || mode == 2);
  const bool unit = (mode == 0 || mode == 3);
  if (lower) {
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      E v = x[r];
#pragma unroll
      for (int c = 0; c < r; ++c) v = fmsc(v, T[r][c], x[c]);
      x[r] = (unit || r >= nb) ? v : el<E>::div(v, T[r][r]);
    }
  } else {
#pragma unroll
    for (int r = NB - 1; r >= 0; --r) {
      E v = x[r];
#pragma unroll
      for (int c = r + 1; c < NB; ++c) v = fmsc(v, T[r][c], x[c]);
      x[r] = (unit || r >= nb) ? v : el<E>::div(v, T[r][r]);
    }
  }
#pragma unroll
  for (int r = 0; r < NB; ++r)
    if (r < nb) B[(long long)(i0 + r) * ldb + col] = x[r];
}

// Many columns overall: one thread per column; few: one warp per column.
template <typename E>
void trsm_diag(cudaStream_t s, const E* A, int lda, long long sA, int i0, int nb, int mode, E* B, int ldb,
               long long sB, int nrhs, int batch) {
  if ((long long)nrhs * batch >= 8192) {
    const int threads = nrhs >= 128 ? 128 : ((nrhs + 31) / 32) * 32;
    dim3 g((nrhs + threads - 1) / threads, batch);
    k_trsm_diag_col<E><<<g, threads, 0, s>>>(A, lda, sA, i0, nb, mode, B, ldb, sB, nrhs);
  } else {
    dim3 g((nrhs + TRSM_WARPS - 1) / TRSM_WARPS, batch);
    k_trsm_diag<E><<<g, 32 * TRSM_WARPS, 0, s>>>(A, lda, sA, i0, nb, mode, B, ldb, sB, nrhs);
  }
  HS_COUNT_LAUNCH();
}

// The solve with a whole diagonal block of up to NBB rows in one launch:
// rows [i0, i0 + nbs) of B (column block of TB_CW<E> columns per CTA, held in
// shared memory) against the block's unit lower (mode 0, top down) or upper
// triangle (mode 1, bottom up).  Per NB-row sub-block: one warp per column
// solves the diagonal block with shuffles, then every thread updates the
// block's remaining rows from the solved ones (the off-diagonal entries read
// through L1).  Replaces the NB-blocked sequence of triangular solves and
// small products (and their trips through global memory) inside the block.
template <typename E> struct tb_cw { static constexpr int v = sizeof(E) == 16 ? 8 : 16; };
template <typename E>
__global__ void __launch_bounds__(32 * tb_cw<E>::v) k_trsm_blk(const E* __restrict__ A, int lda, long long sA, int i0,
                                                               int nbs, int mode, E* __restrict__ B, int ldb,
                                                               long long sB, int nrhs) {
  constexpr int CW = tb_cw<E>::v, NT = 32 * CW;
  __shared__ E Bs[NBB][CW + 1];
  __shared__ E Ld[NB][NB + 1];
  const int b = blockIdx.y, c0 = blockIdx.x * CW, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  A += b * sA;
  B += b * sB;
  for (int e = tid; e < nbs * CW; e += NT) {
    const int r = e / CW, c = e % CW;
    Bs[r][c] = c0 + c < nrhs ? B[(long long)(i0 + r) * ldb + c0 + c] : el<E>::zero();
  }
  const int nsub = (nbs + NB - 1) / NB;
  for (int q = 0; q < nsub; ++q) {
    const int sub = mode == 0 ? q : nsub - 1 - q;
    const int r0 = sub * NB, nb = min(NB, nbs - r0);
    for (int e = tid; e < nb * nb; e += NT) {
      const int r = e / nb, c = e % nb;
      Ld[r][c] = A[(long long)(i0 + r0 + r) * lda + i0 + r0 + c];
    }
    __syncthreads();  // (also orders the previous sub-block's updates of Bs)
    if (warp < CW) {
      E x = lane < nb ? Bs[r0 + lane][warp] : el<E>::zero();
      if (mode == 0) {
        for (int t = 0; t < nb; ++t) {
          const E xt = shfl(x, t);
          if (lane > t && lane < nb) x = fmsc(x, Ld[lane][t], xt);
        }
      } else {
        for (int t = nb - 1; t >= 0; --t) {
          if (lane == t) x = el<E>::div(x, Ld[t][t]);
          const E xt = shfl(x, t);
          if (lane < t) x = fmsc(x, Ld[lane][t], xt);
        }
      }
      if (lane < nb) Bs[r0 + lane][warp] = x;
    }
    __syncthreads();
    // the block's rows still to solve: below (mode 0) or above (mode 1) the sub-block
    const int ra = mode == 0 ? r0 + nb : 0, rb = mode == 0 ? nbs : r0;
    for (int e = tid; e < (rb - ra) * CW; e += NT) {
      const int r = ra + e / CW, c = e % CW;
      const E* arow = A + (long long)(i0 + r) * lda + i0 + r0;
      E acc = Bs[r][c];
      for (int t = 0; t < nb; ++t) acc = fmsc(acc, arow[t], Bs[r0 + t][c]);
      Bs[r][c] = acc;
    }
  }
  __syncthreads();
  for (int e = tid; e < nbs * CW; e += NT) {
    const int r = e / CW, c = e % CW;
    if (c0 + c < nrhs) B[(long long)(i0 + r) * ldb + c0 + c] = Bs[r][c];
  }
}

// Solve with the diagonal block rows [i0, i0 + nbs) of A: one launch of
// k_trsm_blk when there are few columns overall (the root system and the top
// merges, where the NB-blocked sequence is launch- and latency-bound); with
// many (batched leaf and merge systems) the NB-blocked sequence of
// one-thread-per-column solves and products keeps more threads busy.
template <typename E>
void trsm_blk(cudaStream_t s, const E* A, int lda, long long sA, int i0, int nbs, int mode, E* B, int ldb,
              long long sB, int nrhs, int batch) {
  constexpr int CW = tb_cw<E>::v;
  if ((long long)nrhs * batch < 8192) {
    dim3 g((nrhs + CW - 1) / CW, batch);
    k_trsm_blk<E><<<g, 32 * CW, 0, s>>>(A, lda, sA, i0, nbs, mode, B, ldb, sB, nrhs);
    HS_COUNT_LAUNCH();
    return;
  }
  const E m1 = -el<E>::one(), one = el<E>::one();
  const int I1 = i0 + nbs;
  if (mode == 0) {
    for (int j = i0; j < I1; j += NB) {
      const int nb = std::min(NB, I1 - j);
      trsm_diag<E>(s, A, lda, sA, j, nb, 0, B, ldb, sB, nrhs, batch);
      if (I1 - j - nb > 0)
        gemm<E, E, E>(s, OP_N, OP_N, I1 - j - nb, nrhs, nb, m1, A + (long long)(j + nb) * lda + j, lda, sA,
                      B + (long long)j * ldb, ldb, sB, one, B + (long long)(j + nb) * ldb, ldb, sB, batch);
    }
  } else {
    for (int j = i0 + ((nbs - 1) / NB) * NB; j >= i0; j -= NB) {
      const int nb = std::min(NB, I1 - j);
      trsm_diag<E>(s, A, lda, sA, j, nb, 1, B, ldb, sB, nrhs, batch);
      if (j > i0)
        gemm<E, E, E>(s, OP_N, OP_N, j - i0, nrhs, nb, m1, A + (long long)i0 * lda + j, lda, sA,
                      B + (long long)j * ldb, ldb, sB, one, B + (long long)i0 * ldb, ldb, sB, batch);
    }
  }
}

template <typename E>
__global__ void k_swaps(const int* piv, long long sP, int n, int reverse, E* B, int ldb, long long sB, int nrhs) {
  const int b = blockIdx.y;
  piv += b * sP;
  B += b * sB;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= nrhs) return;
  if (!reverse) {
    for (int j = 0; j < n; ++j) {
      int p = piv[j];
      if (p != j) {
        E t = B[(long long)j * ldb + col];
        B[(long long)j * ldb + col] = B[(long long)p * ldb + col];
        B[(long long)p * ldb + col] = t;
      }
    }
  } else {
    for (int j = n - 1; j >= 0; --j) {
      int p = piv[j];
      if (p != j) {
        E t = B[(long long)j * ldb + col];
        B[(long long)j * ldb + col] = B[(long long)p * ldb + col];
        B[(long long)p * ldb + col] = t;
      }
    }
  }
}
}  // namespace

namespace {
// SIMT product (FP64, or FP32 where the tensor-core path is not taken).
template <typename TA, typename TB, typename TC>
void gemm_simt(cudaStream_t s, int opA, int opB, int m, int n, int k, TC alpha, const TA* A, int lda, long long sA,
               const TB* B, int ldb, long long sB, TC beta, TC* C, int ldc, long long sC, int batch) {
  const bool prof = prof_active(is_fp64<TC>::v ? 1 : 2);
  cudaEvent_t ev = nullptr;
  if (prof) prof_begin(s, &ev);
  constexpr long long kFill = 2 * 152;  // tiles that keep every SM of the chip busy
  const long long t64 = (long long)((m + GB - 1) / GB) * ((n + GB - 1) / GB) * batch;
  const long long t32 = (long long)((m + BM - 1) / BM) * ((n + BN - 1) / BN) * batch;
  // 64 x 64 tiles (twice the arithmetic per shared-memory load) when they fill the
  // chip, for matrices of at least one tile each way or with at least 60% of
  // the tiles' outputs inside the matrix (e.g. 56-row blocks)
  const double fill64 = (double)m * n * batch / ((double)t64 * GB * GB);
  // few big tiles with a long k: the same 64 x 64 tiles, k split over a cluster
  int splits64 = 1;
  constexpr bool pipe_types = !is_fp64<TC>::v && sizeof(TA) <= 8 && sizeof(TB) <= 8;
  if (sizeof(TC) <= 8 && t64 < kFill && m >= GB && n >= GB && k >= 256) {
    splits64 = (int)std::min<long long>((kFill + t64 - 1) / t64, k / 128);
    splits64 = std::max(1, std::min(splits64, kMaxCluster));
    if ((long long)batch * splits64 > 65535 || t64 * splits64 < 152) splits64 = 1;
  }
  if ((t64 >= kFill && ((m >= GB && n >= GB) || fill64 >= 0.6)) || splits64 > 1) {
    dim3 grid((n + GB - 1) / GB, (m + GB - 1) / GB, batch * splits64);
    // untransposed FP32 operands with 16-byte aligned rows: the cp.async pipeline
    if constexpr (pipe_types) {
      constexpr int EA = 16 / (int)sizeof(TA), EB = 16 / (int)sizeof(TB);
      const bool aligned = opA == OP_N && opB == OP_N && lda % EA == 0 && ldb % EB == 0 && sA % EA == 0 &&
                           sB % EB == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0 &&
                           (reinterpret_cast<uintptr_t>(B) & 15) == 0;
      if (aligned) {
        constexpr int smem = PipeCfg<TA, TB, TC>::SMEM;
        static bool attr[64] = {};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 0 || dev >= 64 || !attr[dev]) {
          cudaFuncSetAttribute(k_gemm_pipe<TA, TB, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
          if (dev >= 0 && dev < 64) attr[dev] = true;
        }
        if (splits64 == 1) {
          k_gemm_pipe<TA, TB, TC><<<grid, 256, smem, s>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC,
                                                          1);
        } else {
          cudaLaunchConfig_t cfg = {};
          cfg.gridDim = grid;
          cfg.blockDim = dim3(256);
          cfg.dynamicSmemBytes = smem;
          cfg.stream = s;
          cudaLaunchAttribute at[1];
          at[0].id = cudaLaunchAttributeClusterDimension;
          at[0].val.clusterDim.x = 1;
          at[0].val.clusterDim.y = 1;
          at[0].val.clusterDim.z = splits64;
          cfg.attrs = at;
          cfg.numAttrs = 1;
          cudaLaunchKernelEx(&cfg, k_gemm_pipe<TA, TB, TC>, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc,
                             sC, splits64);
        }
        HS_COUNT_LAUNCH();
        if (prof) prof_end(s, ev, flops_per_mac<TA, TB>() * (double)m * n * k * batch);
        return;
      }
    }
    if (splits64 == 1) {
      k_gemm_big<TA, TB, TC><<<grid, 256, 0, s>>>(opA, opB, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC,
                                                  1);
    } else {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = grid;
      cfg.blockDim = dim3(256);
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 1;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = splits64;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      cudaLaunchKernelEx(&cfg, k_gemm_big<TA, TB, TC>, opA, opB, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C,
                         ldc, sC, splits64);
    }
    HS_COUNT_LAUNCH();
  } else {
    int splits = 1;
    if (t32 < kFill && k >= 256) {
      splits = (int)std::min<long long>((kFill + t32 - 1) / t32, k / 128);
      splits = std::max(1, std::min(splits, kMaxCluster));
      if ((long long)batch * splits > 65535) splits = 1;
    }
    dim3 grid((n + BN - 1) / BN, (m + BM - 1) / BM, batch * splits);
    if (splits == 1) {
      k_gemm<TA, TB, TC><<<grid, 256, 0, s>>>(opA, opB, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, 1);
    } else {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = grid;
      cfg.blockDim = dim3(256);
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 1;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = splits;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      cudaLaunchKernelEx(&cfg, k_gemm<TA, TB, TC>, opA, opB, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC,
                         splits);
    }
    HS_COUNT_LAUNCH();
  }
  if (prof) prof_end(s, ev, flops_per_mac<TA, TB>() * (double)m * n * k * batch);
}

// Products the split-TF32 tensor-core path takes (t32_gemm modes): complex x
// complex (2), real x complex (1), real x real (0), FP32, no transposes.
template <typename TA, typename TB, typename TC> struct t32_mode { static constexpr int v = -1; };
template <> struct t32_mode<float2, float2, float2> { static constexpr int v = 2; };
template <> struct t32_mode<float, float2, float2> { static constexpr int v = 1; };
template <> struct t32_mode<float, float, float> { static constexpr int v = 0; };

inline float2 as_f2(float2 x) { return x; }
inline float2 as_f2(float x) { return make_float2(x, 0.f); }
template <typename T> constexpr long long fl() { return sizeof(T) / sizeof(float); }  // floats per element

// Products worth measuring: at least 512 rows and 512 of k in the real
// product, at least 64 columns, and 2^28 real multiply-adds.  Smaller ones
// (the batched leaf, merge and sweep products, the short-k trailing updates)
// never reached the required speed-up over SIMT in the measurements (at most
// 1.4x) and stay there without a measurement, which keeps a frequency sweep,
// whose sizes change from step to step, from paying for one per new shape.
bool t32_candidate(int mode, int m, int n, int k, int batch) {
  const long long np = mode ? 2LL * n : n, kp = mode == 2 ? 2LL * k : k;
  return m >= 512 && np >= 64 && kp >= 512 && (long long)m * np * kp * batch >= (1LL << 28);
}

// Per-shape choice between the tensor-core and the SIMT product, measured
// once per shape class (both variants on a scratch copy of C, CUDA events,
// best of two after a warm-up) outside stream capture; inside a capture a
// shape not yet measured takes the default.
// Shapes are keyed in half-octave classes (a frequency sweep changes its sizes
// in small steps; one measurement serves a class).
inline int size_class(long long x) { return x <= 1 ? 0 : (int)std::lround(2.0 * std::log2((double)x)); }
struct TuneKey {
  int mode, m, n, k, batch, bsh;
  bool operator<(const TuneKey& o) const {
    return std::tie(mode, m, n, k, batch, bsh) < std::tie(o.mode, o.m, o.n, o.k, o.batch, o.bsh);
  }
};

std::mutex g_tune_mu;
std::map<TuneKey, bool> g_tune;

}  // namespace

bool g_autotune = true;             // hs_set_autotune
// The tensor-core product's accumulation is coarser than SIMT FMA chains, which
// slows the refinement of the mixed solver; it is kept only where it takes
// less than half the SIMT time (hs_set_tc_margin).
float g_tc_margin = 0.5f;
int g_t32_mode = 1;                 // hs_set_tensor_cores: 0 off, 1 per-shape choice, 2 forced
thread_local bool g_prof_suspended = false;
thread_local int g_last_gemm_tc = 0;

template <typename TA, typename TB, typename TC>
void gemm(cudaStream_t s, int opA, int opB, int m, int n, int k, TC alpha, const TA* A, int lda, long long sA,
          const TB* B, int ldb, long long sB, TC beta, TC* C, int ldc, long long sC, int batch) {
  if (m <= 0 || n <= 0 || batch <= 0) return;
  g_last_gemm_tc = 0;
  constexpr int mode = t32_mode<TA, TB, TC>::v;
  if constexpr (mode >= 0) {
    const bool force = g_t32_mode == 2;
    if (opA == OP_N && opB == OP_N && k > 0 && g_t32_mode != 0 && (force || t32_candidate(mode, m, n, k, batch))) {
      auto run_tc = [&](TC* Cd) {
        return t32_gemm(s, mode, m, n, k, as_f2(alpha), reinterpret_cast<const float*>(A), fl<TA>() * lda,
                        fl<TA>() * sA, reinterpret_cast<const float*>(B), fl<TB>() * ldb, fl<TB>() * sB, as_f2(beta),
                        Cd, ldc, sC, batch);
      };
      bool use = true;  // forced, or a candidate not yet measured inside a capture
      const TuneKey key{mode, size_class(m), size_class(n), size_class(k), size_class(batch),
                        (sB == 0 && batch > 1) ? 1 : 0};
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      cudaStreamIsCapturing(s, &cs);
      bool known = false;
      {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end() && !force) {
          use = it->second;
          known = true;
        }
      }
      if (!known && !force && g_autotune && cs == cudaStreamCaptureStatusNone) {
        // measure both on a copy of C (the real C is written once, below)
        const long long span = (long long)(batch - 1) * sC + (long long)(m - 1) * ldc + n;
        TC* tmp = nullptr;
        if (cudaMalloc(&tmp, sizeof(TC) * span) == cudaSuccess) {
          long long* counter = g_launch_counter;
          g_launch_counter = nullptr;
          g_prof_suspended = true;
          cudaEvent_t ev[3];
          for (auto& e : ev) cudaEventCreate(&e);
          float best_tc = 1e30f, best_simt = 1e30f;
          bool tc_ok = true;
          for (int rep = 0; rep < 3 && tc_ok; ++rep) {
            cudaMemcpyAsync(tmp, C, sizeof(TC) * span, cudaMemcpyDeviceToDevice, s);
            cudaEventRecord(ev[0], s);
            tc_ok = run_tc(tmp);
            cudaEventRecord(ev[1], s);
            gemm_simt<TA, TB, TC>(s, opA, opB, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, tmp, ldc, sC, batch);
            cudaEventRecord(ev[2], s);
            cudaEventSynchronize(ev[2]);
            float t1 = 0.f, t2 = 0.f;
            cudaEventElapsedTime(&t1, ev[0], ev[1]);
            cudaEventElapsedTime(&t2, ev[1], ev[2]);
            if (rep > 0) {
              best_tc = std::min(best_tc, t1);
              best_simt = std::min(best_simt, t2);
            }
          }
          for (auto& e : ev) cudaEventDestroy(e);
          cudaFree(tmp);
          g_prof_suspended = false;
          g_launch_counter = counter;
          use = tc_ok && best_tc < g_tc_margin * best_simt;
          std::lock_guard<std::mutex> lock(g_tune_mu);
          g_tune[key] = use;
        } else {
          cudaGetLastError();
        }
      }
      if (use && run_tc(C)) {
        g_last_gemm_tc = 1;
        return;
      }
    }
  }
  gemm_simt<TA, TB, TC>(s, opA, opB, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch);
}

template <typename E>
void lu_factor(cudaStream_t s, E* A, int lda, long long sA, int n, int* piv, long long sP, int* info, int batch) {
  const E m1 = -el<E>::one(), one = el<E>::one();
  // Two-level right-looking blocking: super-panels of NBB columns, each
  // factored as NB-wide pivoted panels whose updates stay inside the
  // super-panel; then U12 = L11^-1 A12 for the super-panel's rows and one
  // trailing update with k = NBB (the product the tensor cores take).
  for (int J0 = 0; J0 < n; J0 += NBB) {
    const int nbs = std::min(NBB, n - J0), J1 = J0 + nbs;
    for (int j0 = J0; j0 < J1; j0 += NB) {
      const int nb = std::min(NB, J1 - j0);
      lu_panel<E>(s, A, lda, sA, n, j0, nb, piv, sP, info, batch);  // row moves cover every column
      const int rin = J1 - j0 - nb;  // columns of the super-panel right of this panel
      if (rin > 0) {
        trsm_diag<E>(s, A, lda, sA, j0, nb, 0, A + j0 + nb, lda, sA, rin, batch);
        gemm<E, E, E>(s, OP_N, OP_N, n - j0 - nb, rin, nb, m1, A + (long long)(j0 + nb) * lda + j0, lda, sA,
                      A + (long long)j0 * lda + j0 + nb, lda, sA, one, A + (long long)(j0 + nb) * lda + j0 + nb, lda,
                      sA, batch);
      }
    }
    const int rest = n - J1;
    if (rest > 0) {
      trsm_blk<E>(s, A, lda, sA, J0, nbs, 0, A + J1, lda, sA, rest, batch);  // U12 = L11^-1 A12
      gemm<E, E, E>(s, OP_N, OP_N, rest, rest, nbs, m1, A + (long long)J1 * lda + J0, lda, sA,
                    A + (long long)J0 * lda + J1, lda, sA, one, A + (long long)J1 * lda + J1, lda, sA, batch);
    }
  }
}

namespace {
template <typename E> __global__ void k_identity(E* A, int n, int lda, long long sA) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int r = (int)(e / n), c = (int)(e % n);
  A[blockIdx.y * sA + (long long)r * lda + c] = r == c ? el<E>::one() : el<E>::zero();
}
}  // namespace

template <typename E>
void lu_inverse(cudaStream_t s, const E* A, int lda, long long sA, int n, const int* piv, long long sP, E* Inv,
                int ldi, long long sI, int batch) {
  dim3 g((unsigned)(((long long)n * n + 255) / 256), batch);
  k_identity<E><<<g, 256, 0, s>>>(Inv, n, ldi, sI);
  HS_COUNT_LAUNCH();
  lu_solve<E>(s, OP_N, A, lda, sA, n, piv, sP, Inv, ldi, sI, n, batch);
}

template <typename E>
void lu_solve(cudaStream_t s, int trans, const E* A, int lda, long long sA, int n, const int* piv, long long sP, E* B,
              int ldb, long long sB, int nrhs, int batch) {
  dim3 gs((nrhs + 127) / 128, batch);
  const E m1 = -el<E>::one(), one = el<E>::one();
  if (trans == OP_N) {
    k_swaps<E><<<gs, 128, 0, s>>>(piv, sP, n, 0, B, ldb, sB, nrhs);
    HS_COUNT_LAUNCH();
    // blocks of NBB rows (one launch solves a block's diagonal triangle),
    // then one update of the remaining rows with k = NBB
    for (int I0 = 0; I0 < n; I0 += NBB) {  // L y = b
      const int I1 = std::min(n, I0 + NBB);
      trsm_blk<E>(s, A, lda, sA, I0, I1 - I0, 0, B, ldb, sB, nrhs, batch);
      if (n - I1 > 0)
        gemm<E, E, E>(s, OP_N, OP_N, n - I1, nrhs, I1 - I0, m1, A + (long long)I1 * lda + I0, lda, sA,
                      B + (long long)I0 * ldb, ldb, sB, one, B + (long long)I1 * ldb, ldb, sB, batch);
    }
    const int lastB = ((n - 1) / NBB) * NBB;
    for (int I0 = lastB; I0 >= 0; I0 -= NBB) {  // U x = y
      const int I1 = std::min(n, I0 + NBB);
      trsm_blk<E>(s, A, lda, sA, I0, I1 - I0, 1, B, ldb, sB, nrhs, batch);
      if (I0 > 0)
        gemm<E, E, E>(s, OP_N, OP_N, I0, nrhs, I1 - I0, m1, A + I0, lda, sA, B + (long long)I0 * ldb, ldb, sB, one, B,
                      ldb, sB, batch);
    }
  } else {
    for (int i0 = 0; i0 < n; i0 += NB) {  // U^T y = b
      int nb = n - i0 < NB ? n - i0 : NB;
      trsm_diag<E>(s, A, lda, sA, i0, nb, 2, B, ldb, sB, nrhs, batch);
      int rest = n - i0 - nb;
      if (rest > 0)
        gemm<E, E, E>(s, OP_T, OP_N, rest, nrhs, nb, m1, A + (long long)i0 * lda + i0 + nb, lda, sA,
                      B + (long long)i0 * ldb, ldb, sB, one, B + (long long)(i0 + nb) * ldb, ldb, sB, batch);
    }
    int last = ((n - 1) / NB) * NB;
    for (int i0 = last; i0 >= 0; i0 -= NB) {  // L^T w = y
      int nb = n - i0 < NB ? n - i0 : NB;
      trsm_diag<E>(s, A, lda, sA, i0, nb, 3, B, ldb, sB, nrhs, batch);
      if (i0 > 0)
        gemm<E, E, E>(s, OP_T, OP_N, i0, nrhs, nb, m1, A + (long long)i0 * lda, lda, sA, B + (long long)i0 * ldb, ldb,
                      sB, one, B, ldb, sB, batch);
    }
    k_swaps<E><<<gs, 128, 0, s>>>(piv, sP, n, 1, B, ldb, sB, nrhs);
    HS_COUNT_LAUNCH();
  }
}

// explicit instantiations
template void gemm<double, double, double>(cudaStream_t, int, int, int, int, int, double, const double*, int,
                                           long long, const double*, int, long long, double, double*, int, long long,
                                           int);
template void gemm<double2, double2, double2>(cudaStream_t, int, int, int, int, int, double2, const double2*, int,
                                              long long, const double2*, int, long long, double2, double2*, int,
                                              long long, int);
template void gemm<double, double2, double2>(cudaStream_t, int, int, int, int, int, double2, const double*, int,
                                             long long, const double2*, int, long long, double2, double2*, int,
                                             long long, int);
template void gemm<double2, double, double2>(cudaStream_t, int, int, int, int, int, double2, const double2*, int,
                                             long long, const double*, int, long long, double2, double2*, int,
                                             long long, int);
template void lu_factor<double>(cudaStream_t, double*, int, long long, int, int*, long long, int*, int);
template void lu_factor<double2>(cudaStream_t, double2*, int, long long, int, int*, long long, int*, int);
template void lu_solve<double>(cudaStream_t, int, const double*, int, long long, int, const int*, long long, double*,
                               int, long long, int, int);
template void lu_solve<double2>(cudaStream_t, int, const double2*, int, long long, int, const int*, long long,
                                double2*, int, long long, int, int);

template void gemm<float, float, float>(cudaStream_t, int, int, int, int, int, float, const float*, int, long long,
                                        const float*, int, long long, float, float*, int, long long, int);
template void gemm<float2, float2, float2>(cudaStream_t, int, int, int, int, int, float2, const float2*, int,
                                           long long, const float2*, int, long long, float2, float2*, int, long long,
                                           int);
template void gemm<float, float2, float2>(cudaStream_t, int, int, int, int, int, float2, const float*, int, long long,
                                          const float2*, int, long long, float2, float2*, int, long long, int);
template void gemm<float2, float, float2>(cudaStream_t, int, int, int, int, int, float2, const float2*, int,
                                          long long, const float*, int, long long, float2, float2*, int, long long,
                                          int);
template void lu_factor<float>(cudaStream_t, float*, int, long long, int, int*, long long, int*, int);
template void lu_factor<float2>(cudaStream_t, float2*, int, long long, int, int*, long long, int*, int);
template void lu_inverse<double>(cudaStream_t, const double*, int, long long, int, const int*, long long, double*, int,
                                 long long, int);
template void lu_inverse<float>(cudaStream_t, const float*, int, long long, int, const int*, long long, float*, int,
                                long long, int);
template void lu_inverse<float2>(cudaStream_t, const float2*, int, long long, int, const int*, long long, float2*, int,
                                 long long, int);
template void lu_solve<float>(cudaStream_t, int, const float*, int, long long, int, const int*, long long, float*, int,
                              long long, int, int);
template void lu_solve<float2>(cudaStream_t, int, const float2*, int, long long, int, const int*, long long, float2*,
                               int, long long, int, int);

}  // namespace hs
