// Shared device/host helpers for libhs: complex arithmetic on double2/float2,
// error propagation and launch bookkeeping.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

namespace hs {

// ---- complex arithmetic (interleaved re/im, same layout as the C ABI) ------
struct Cz { double x, y; };   // complex double, 16-byte aligned like double2

__host__ __device__ inline double2 cz(double re, double im) { return make_double2(re, im); }
__host__ __device__ inline double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 operator-(double2 a) { return make_double2(-a.x, -a.y); }
__host__ __device__ inline double2 operator*(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__host__ __device__ inline double2 operator*(double2 a, double s) { return make_double2(s * a.x, s * a.y); }
__host__ __device__ inline double2 conjz(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ inline double abs2z(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ inline double2 divz(double2 a, double2 b) {
  // Smith's algorithm (avoids overflow for large |b|).
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  } else {
    double r = b.x / b.y, d = b.y + b.x * r;
    return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
  }
}

// complex float (FP32 factors of the mixed-precision path)
__host__ __device__ inline float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline float2 operator-(float2 a) { return make_float2(-a.x, -a.y); }
__host__ __device__ inline float2 operator*(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__host__ __device__ inline float abs2z(float2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ inline float2 divz(float2 a, float2 b) {
  if (fabsf(b.x) >= fabsf(b.y)) {
    float r = b.y / b.x, d = b.x + b.y * r;
    return make_float2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  } else {
    float r = b.x / b.y, d = b.y + b.x * r;
    return make_float2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
  }
}

// Generic element traits so that the linear algebra can be templated on
// real or complex element types.
template <typename E> struct el;
template <> struct el<double> {
  __host__ __device__ static double zero() { return 0.0; }
  __host__ __device__ static double one() { return 1.0; }
  __host__ __device__ static double mag2(double a) { return a * a; }
  __host__ __device__ static double div(double a, double b) { return a / b; }
};
template <> struct el<double2> {
  __host__ __device__ static double2 zero() { return make_double2(0.0, 0.0); }
  __host__ __device__ static double2 one() { return make_double2(1.0, 0.0); }
  __host__ __device__ static double mag2(double2 a) { return abs2z(a); }
  __host__ __device__ static double2 div(double2 a, double2 b) { return divz(a, b); }
};
template <> struct el<float> {
  __host__ __device__ static float zero() { return 0.0f; }
  __host__ __device__ static float one() { return 1.0f; }
  __host__ __device__ static double mag2(float a) { return (double)a * a; }
  __host__ __device__ static float div(float a, float b) { return a / b; }
};
template <> struct el<float2> {
  __host__ __device__ static float2 zero() { return make_float2(0.0f, 0.0f); }
  __host__ __device__ static float2 one() { return make_float2(1.0f, 0.0f); }
  __host__ __device__ static double mag2(float2 a) { return (double)abs2z(a); }
  __host__ __device__ static float2 div(float2 a, float2 b) { return divz(a, b); }
};

// Real and complex types of one precision.
template <typename T> struct prec;
template <> struct prec<double> { using R = double; using C = double2; };
template <> struct prec<float> { using R = float; using C = float2; };
__host__ __device__ inline double2 to_c(double2 a, double2*) { return a; }
__host__ __device__ inline float2 to_c(double2 a, float2*) { return make_float2((float)a.x, (float)a.y); }
__host__ __device__ inline double2 to_c(float2 a, double2*) { return make_double2(a.x, a.y); }
__host__ __device__ inline float2 to_c(float2 a, float2*) { return a; }
template <typename C, typename S> __host__ __device__ inline C cvt(S a) { return to_c(a, (C*)nullptr); }

// Mixed-type multiply-accumulate used by the GEMM templates.
__host__ __device__ inline double mul(double a, double b) { return a * b; }
__host__ __device__ inline double2 mul(double a, double2 b) { return make_double2(a * b.x, a * b.y); }
__host__ __device__ inline double2 mul(double2 a, double b) { return make_double2(a.x * b, a.y * b); }
__host__ __device__ inline double2 mul(double2 a, double2 b) { return a * b; }
__host__ __device__ inline bool is_zero(double a) { return a == 0.0; }
__host__ __device__ inline bool is_zero(double2 a) { return a.x == 0.0 && a.y == 0.0; }
__host__ __device__ inline double addv(double a, double b) { return a + b; }
__host__ __device__ inline double2 addv(double2 a, double2 b) { return a + b; }
template <typename TC, typename S> __host__ __device__ inline TC scal(S s, TC v);
template <> __host__ __device__ inline double scal<double, double>(double s, double v) { return s * v; }
template <> __host__ __device__ inline double2 scal<double2, double2>(double2 s, double2 v) { return s * v; }
__host__ __device__ inline float mul(float a, float b) { return a * b; }
__host__ __device__ inline float2 mul(float a, float2 b) { return make_float2(a * b.x, a * b.y); }
__host__ __device__ inline float2 mul(float2 a, float b) { return make_float2(a.x * b, a.y * b); }
__host__ __device__ inline float2 mul(float2 a, float2 b) { return a * b; }
__host__ __device__ inline bool is_zero(float a) { return a == 0.0f; }
__host__ __device__ inline bool is_zero(float2 a) { return a.x == 0.0f && a.y == 0.0f; }
__host__ __device__ inline float addv(float a, float b) { return a + b; }
__host__ __device__ inline float2 addv(float2 a, float2 b) { return a + b; }
template <> __host__ __device__ inline float scal<float, float>(float s, float v) { return s * v; }

// acc + a b with one fused multiply-add per real product (4 for complex x
// complex instead of 2 products, 1 product-sum and 2 additions): the FP64
// pipe is the binding resource of the GEMM kernels.
__host__ __device__ inline double fmac(double acc, double a, double b) { return fma(a, b, acc); }
__host__ __device__ inline double2 fmac(double2 acc, double a, double2 b) {
  return make_double2(fma(a, b.x, acc.x), fma(a, b.y, acc.y));
}
__host__ __device__ inline double2 fmac(double2 acc, double2 a, double b) {
  return make_double2(fma(a.x, b, acc.x), fma(a.y, b, acc.y));
}
__host__ __device__ inline double2 fmac(double2 acc, double2 a, double2 b) {
  return make_double2(fma(-a.y, b.y, fma(a.x, b.x, acc.x)), fma(a.y, b.x, fma(a.x, b.y, acc.y)));
}
__host__ __device__ inline float fmac(float acc, float a, float b) { return fmaf(a, b, acc); }
__host__ __device__ inline float2 fmac(float2 acc, float a, float2 b) {
  return make_float2(fmaf(a, b.x, acc.x), fmaf(a, b.y, acc.y));
}
__host__ __device__ inline float2 fmac(float2 acc, float2 a, float b) {
  return make_float2(fmaf(a.x, b, acc.x), fmaf(a.y, b, acc.y));
}
__host__ __device__ inline float2 fmac(float2 acc, float2 a, float2 b) {
  return make_float2(fmaf(-a.y, b.y, fmaf(a.x, b.x, acc.x)), fmaf(a.y, b.x, fmaf(a.x, b.y, acc.y)));
}
// acc - a b, fused the same way
__host__ __device__ inline double fmsc(double acc, double a, double b) { return fma(-a, b, acc); }
__host__ __device__ inline double2 fmsc(double2 acc, double2 a, double2 b) {
  return make_double2(fma(a.y, b.y, fma(-a.x, b.x, acc.x)), fma(-a.y, b.x, fma(-a.x, b.y, acc.y)));
}
__host__ __device__ inline float fmsc(float acc, float a, float b) { return fmaf(-a, b, acc); }
__host__ __device__ inline float2 fmsc(float2 acc, float2 a, float2 b) {
  return make_float2(fmaf(a.y, b.y, fmaf(-a.x, b.x, acc.x)), fmaf(-a.y, b.x, fmaf(-a.x, b.y, acc.y)));
}
template <> __host__ __device__ inline float2 scal<float2, float2>(float2 s, float2 v) { return s * v; }

}  // namespace hs

// Launch bookkeeping: every kernel launch in the library goes through HS_LAUNCH
// so that the context can report how many of its kernels ran.
namespace hs {
extern thread_local long long* g_launch_counter;
}
#define HS_COUNT_LAUNCH()                        \
  do {                                           \
    if (hs::g_launch_counter) ++(*hs::g_launch_counter); \
  } while (0)

// Named phase of the host orchestration, visible to profilers (NVTX range).
namespace hs {
struct Phase {
  explicit Phase(const char* name) { nvtxRangePushA(name); }
  ~Phase() { nvtxRangePop(); }
};
}  // namespace hs
