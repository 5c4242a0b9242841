// Measurement hooks (include/hs_diag.h): per-launch timing of the FP64 GEMM
// family and an FP64 DFMA peak kernel.
#include <vector>

#include "../../include/hs.h"
#include "../../include/hs_diag.h"
#include "common.cuh"
#include "linalg.cuh"
#include "tree.cuh"

namespace hs {

struct ProfRec {
  cudaEvent_t a, b;
  double flops;
};

namespace {
int g_prof_family = 0;
std::vector<ProfRec> g_prof;
}  // namespace

bool prof_active(int family) { return !g_prof_suspended && g_prof_family == family; }
bool prof_any() { return g_prof_family != 0; }
extern bool g_use_graphs;
extern size_t g_contract_budget;
extern int g_fail_allocs;

void prof_begin(cudaStream_t s, cudaEvent_t* a) {
  cudaEventCreate(a);
  cudaEventRecord(*a, s);
}

void prof_end(cudaStream_t s, cudaEvent_t a, double flops) {
  ProfRec r;
  r.a = a;
  cudaEventCreate(&r.b);
  cudaEventRecord(r.b, s);
  r.flops = flops;
  g_prof.push_back(r);
}

// Independent DFMA chains: 8 accumulators per thread, `iters` rounds.
__global__ void k_dfma_peak(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-9, x1 = x0 + 1e-9, x2 = x0 + 2e-9, x3 = x0 + 3e-9;
  double x4 = x0 + 4e-9, x5 = x0 + 5e-9, x6 = x0 + 6e-9, x7 = x0 + 7e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  double s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == 12345.678) out[0] = s;  // keeps the chains live
}

// The same with FP32 FFMA chains (16 accumulators per thread).
__global__ void k_ffma_peak(float* out, int iters, float a, float b) {
  float x[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) x[j] = threadIdx.x * 1e-6f + j * 1e-6f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int j = 0; j < 16; ++j) x[j] = fmaf(x[j], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 16; ++j) s += x[j];
  if (s == 12345.678f) out[0] = s;  // keeps the chains live
}

// Time `kern` (k_dfma_peak or k_ffma_peak) for about `ms`: returns the
// measured milliseconds and the iteration count it ran with.
template <typename T, typename K>
float time_peak(K kern, T* out, int blocks, int threads, double ms, T a, T b, int* iters_out) {
  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  int iters = 256;
  float t = 0.f;
  for (int rep = 0; rep < 6; ++rep) {  // warm up and scale the iteration count to the requested duration
    cudaEventRecord(ev0);
    kern<<<blocks, threads>>>(out, iters, a, b);
    cudaEventRecord(ev1);
    cudaEventSynchronize(ev1);
    cudaEventElapsedTime(&t, ev0, ev1);
    if (t > 0.5 * ms) break;
    iters *= 2;
  }
  cudaEventRecord(ev0);
  kern<<<blocks, threads>>>(out, iters, a, b);
  cudaEventRecord(ev1);
  cudaEventSynchronize(ev1);
  cudaEventElapsedTime(&t, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  *iters_out = iters;
  return t;
}

}  // namespace hs

extern "C" {

int hs_peak_fp32(int device, double ms, double* tflops) {
  if (!tflops || !(ms > 0)) return HS_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return HS_ECUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float)) != cudaSuccess) return HS_ENOMEM;
  const int threads = 256, blocks = sms * 8;
  int iters = 0;
  const float t = hs::time_peak<float>(hs::k_ffma_peak, out, blocks, threads, ms, 0.9999999f, 1e-7f, &iters);
  const double ffma = (double)blocks * threads * iters * 8.0 * 16.0;
  *tflops = 2.0 * ffma / (t * 1e-3) / 1e12;
  cudaFree(out);
  return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ECUDA;
}

int hs_prof_start(int family) {
  if (family != HS_PROF_GEMM_FP64 && family != HS_PROF_GEMM_FP32 && family != HS_PROF_GEMM_TC &&
      family != HS_PROF_GEMM_EMU)
    return HS_EINVAL;
  hs::g_prof.clear();
  hs::g_prof_family = family;
  return HS_OK;
}

int hs_prof_stop(double* total_ms, double* total_flops, long long* launches) {
  hs::g_prof_family = 0;
  double ms = 0.0, fl = 0.0;
  for (auto& r : hs::g_prof) {
    cudaEventSynchronize(r.b);
    float t = 0.f;
    cudaEventElapsedTime(&t, r.a, r.b);
    ms += t;
    fl += r.flops;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  long long n = (long long)hs::g_prof.size();
  hs::g_prof.clear();
  if (total_ms) *total_ms = ms;
  if (total_flops) *total_flops = fl;
  if (launches) *launches = n;
  return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ECUDA;
}

int hs_peak_fp64(int device, double ms, double* tflops) {
  if (!tflops || !(ms > 0)) return HS_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return HS_ECUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return HS_ENOMEM;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int threads = 256, blocks = sms * 8;
  int iters = 256;
  float t = 0.f;
  // warm up and scale the iteration count to the requested duration
  for (int rep = 0; rep < 6; ++rep) {
    cudaEventRecord(a);
    hs::k_dfma_peak<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&t, a, b);
    if (t > 0.5 * ms) break;
    iters = (int)(iters * 2);
  }
  cudaEventRecord(a);
  hs::k_dfma_peak<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
  cudaEventRecord(b);
  cudaEventSynchronize(b);
  cudaEventElapsedTime(&t, a, b);
  double dfma = (double)blocks * threads * iters * 16.0 * 8.0;
  *tflops = 2.0 * dfma / (t * 1e-3) / 1e12;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ECUDA;
}

int hs_set_graphs(int enable) {
  hs::g_use_graphs = enable != 0;
  return HS_OK;
}

int hs_set_contract_budget(unsigned long long bytes) {
  hs::g_contract_budget = bytes ? (size_t)bytes : (size_t(1) << 30);
  return HS_OK;
}

int hs_set_fp64_emulation(int enable) {
  hs::g_oz_enabled = enable != 0;
  return HS_OK;
}

int hs_dgemm_emulated(int m, int n, int k, const void* A, const void* B, void* C, int batch, void* stream) {
  if (m <= 0 || n <= 0 || k <= 0 || batch <= 0 || batch > 65535 || !A || !B || !C) return HS_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double* a = const_cast<double*>(static_cast<const double*>(A));
  double* b = const_cast<double*>(static_cast<const double*>(B));
  // A(b, i, kk) = A[b m k + i k + kk];  Bt(b, j, kk) = B[b k n + kk n + j];  C(b, i, j) = C[b m n + i n + j]
  const hs::OzView va{a, (long long)m * k, k, 0, 1, 1}, vb{b, (long long)k * n, 1, 0, n, 1},
      vc{static_cast<double*>(C), (long long)m * n, n, 0, 1, 1};
  const size_t bytes = hs::ozaki_scratch_bytes(m, n, k, batch, false);
  void* scratch = nullptr;
  if (cudaMallocAsync(&scratch, bytes, s) != cudaSuccess) return HS_ENOMEM;
  const cudaError_t e = hs::ozaki_gemm(s, m, n, k, batch, 1.0, va, vb, false, 0.0, vc, scratch, bytes);
  cudaFreeAsync(scratch, s);
  if (e == cudaErrorNotSupported) return HS_ECUDA;
  if (e != cudaSuccess) return e == cudaErrorInvalidValue ? HS_EINVAL : HS_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return HS_ECUDA;
  if (hs::tc_timed_out(s)) return HS_ETIMEOUT;
  return HS_OK;
}

int hs_fail_next_allocs(int n) {
  if (n < 0) return HS_EINVAL;
  hs::g_fail_allocs = n;
  return HS_OK;
}

int hs_raise_tc_timeout(int device) {
  if (cudaSetDevice(device) != cudaSuccess) return HS_ECUDA;
  return hs::tc_raise_timeout_flag() == cudaSuccess ? HS_OK : HS_ECUDA;
}

int hs_set_tensor_cores(int enable) {
  if (enable < 0 || enable > 2) return HS_EINVAL;
  hs::g_t32_mode = enable;
  return HS_OK;
}

int hs_set_autotune(int enable) {
  hs::g_autotune = enable != 0;
  return HS_OK;
}

int hs_set_tc_margin(double margin) {
  if (!(margin > 0.0 && margin <= 1.0)) return HS_EINVAL;
  hs::g_tc_margin = (float)margin;
  return HS_OK;
}

int hs_gemm32(int mode, int m, int n, int k, const void* A, const void* B, void* C, int batch, int b_shared,
              void* stream, int* used_tc) {
  if (mode < 0 || mode > 2 || m <= 0 || n <= 0 || k <= 0 || batch <= 0 || batch > 65535 || !A || !B || !C)
    return HS_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const long long sB = b_shared ? 0 : (long long)k * n;
  if (mode == 2) {
    hs::gemm<float2, float2, float2>(s, hs::OP_N, hs::OP_N, m, n, k, make_float2(1.f, 0.f),
                                     static_cast<const float2*>(A), k, (long long)m * k, static_cast<const float2*>(B),
                                     n, sB, make_float2(0.f, 0.f), static_cast<float2*>(C), n, (long long)m * n,
                                     batch);
  } else if (mode == 1) {
    hs::gemm<float, float2, float2>(s, hs::OP_N, hs::OP_N, m, n, k, make_float2(1.f, 0.f),
                                    static_cast<const float*>(A), k, (long long)m * k, static_cast<const float2*>(B),
                                    n, sB, make_float2(0.f, 0.f), static_cast<float2*>(C), n, (long long)m * n, batch);
  } else {
    hs::gemm<float, float, float>(s, hs::OP_N, hs::OP_N, m, n, k, 1.f, static_cast<const float*>(A), k,
                                  (long long)m * k, static_cast<const float*>(B), n, sB, 0.f, static_cast<float*>(C),
                                  n, (long long)m * n, batch);
  }
  if (used_tc) *used_tc = hs::g_last_gemm_tc;
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return HS_ECUDA;
  if (hs::tc_timed_out(s)) return HS_ETIMEOUT;
  return HS_OK;
}

int hs_cgemm32(int m, int n, int k, const void* A, const void* B, void* C, int batch, void* stream, int* used_tc) {
  if (m <= 0 || n <= 0 || k <= 0 || batch <= 0 || batch > 65535 || !A || !B || !C) return HS_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  hs::gemm<float2, float2, float2>(s, hs::OP_N, hs::OP_N, m, n, k, make_float2(1.f, 0.f),
                                   static_cast<const float2*>(A), k, (long long)m * k,
                                   static_cast<const float2*>(B), n, (long long)k * n, make_float2(0.f, 0.f),
                                   static_cast<float2*>(C), n, (long long)m * n, batch);
  if (used_tc) *used_tc = hs::g_last_gemm_tc;
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return HS_ECUDA;
  if (hs::tc_timed_out(s)) return HS_ETIMEOUT;
  return HS_OK;
}

int hs_zgemm(int transA, int transB, int m, int n, int k, const void* A, const void* B, void* C, int accumulate,
             void* stream) {
  if (m <= 0 || n <= 0 || k <= 0 || !A || !B || !C) return HS_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int opA = transA ? hs::OP_T : hs::OP_N, opB = transB ? hs::OP_T : hs::OP_N;
  hs::gemm<double2, double2, double2>(s, opA, opB, m, n, k, make_double2(1.0, 0.0), static_cast<const double2*>(A),
                                      transA ? m : k, 0, static_cast<const double2*>(B), transB ? k : n, 0,
                                      make_double2(accumulate ? 1.0 : 0.0, 0.0), static_cast<double2*>(C), n, 0, 1);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return HS_ECUDA;
  return HS_OK;
}

int hs_lu_solve(int precision, int n, int nrhs, void* A, void* B, int batch, void* stream) {
  if (n <= 0 || nrhs <= 0 || batch <= 0 || batch > 65535 || !A || !B) return HS_EINVAL;
  if (precision != HS_FP64 && precision != HS_MIXED) return HS_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int *piv = nullptr, *info = nullptr;
  if (cudaMalloc(&piv, sizeof(int) * (size_t)n * batch) != cudaSuccess) return HS_ENOMEM;
  if (cudaMalloc(&info, sizeof(int) * (size_t)batch) != cudaSuccess) {
    cudaFree(piv);
    return HS_ENOMEM;
  }
  cudaMemsetAsync(info, 0, sizeof(int) * (size_t)batch, s);
  const long long sA = (long long)n * n, sB = (long long)n * nrhs;
  if (precision == HS_FP64) {
    hs::lu_factor<double2>(s, static_cast<double2*>(A), n, sA, n, piv, n, info, batch);
    hs::lu_solve<double2>(s, hs::OP_N, static_cast<double2*>(A), n, sA, n, piv, n, static_cast<double2*>(B), nrhs, sB,
                          nrhs, batch);
  } else {
    hs::lu_factor<float2>(s, static_cast<float2*>(A), n, sA, n, piv, n, info, batch);
    hs::lu_solve<float2>(s, hs::OP_N, static_cast<float2*>(A), n, sA, n, piv, n, static_cast<float2*>(B), nrhs, sB,
                         nrhs, batch);
  }
  std::vector<int> h(batch);
  cudaError_t e = cudaMemcpyAsync(h.data(), info, sizeof(int) * (size_t)batch, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(piv);
  cudaFree(info);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return HS_ECUDA;
  for (int v : h)
    if (v != 0) return HS_ESINGULAR;
  return HS_OK;
}

int hs_jacobian32_products(long long rows, int n, const void* J, const double* v, void* y, const void* u, double* g,
                           void* stream) {
  if (rows <= 0 || n <= 0 || hs::gemvT_parts(rows) > 65535 || !J || !v || !y || !u || !g) return HS_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double* part = nullptr;
  if (cudaMalloc(&part, sizeof(double) * (size_t)hs::gemvT_parts(rows) * n) != cudaSuccess) return HS_ENOMEM;
  const float2* J32 = static_cast<const float2*>(J);
  hs::gemv32(s, J32, rows, n, v, static_cast<double2*>(y));
  hs::gemvT32(s, J32, rows, n, static_cast<const double2*>(u), part, g);
  const cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(part);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return HS_ECUDA;
  return HS_OK;
}

}  // extern "C"
