// Allocation-free far-field solve (hs_solve_noalloc in include/hs.h).
//
// Some callers cannot let the library call cudaMalloc while they run: their
// device memory is owned by another allocator (a framework's caching pool or a
// fixed arena reserved at start-up), so an allocation behind their back breaks
// their accounting or exceeds their cap.  For them the far-field solve takes
// its temporaries from one static device array of fixed size instead of the
// context's growable workspace.  The array lives in this translation unit;
// host code only ever uses its device address, looked up once per device.
#include <mutex>

#include "../../include/hs.h"
#include "common.cuh"

namespace hs {
int ctx_device(const hs_ctx* ctx);
int solve_far_in_scratch(hs_ctx* ctx, void* stream, const double* alphas, int M, const double* thetas, int P,
                         double* ufar, void* scratch, size_t scratch_bytes);
}  // namespace hs

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB on every device that loads libhs
constexpr int kMaxDevices = 64;

// The scratch.  In host code this name is a host-side stand-in for the device
// object, not a device address: never hand it to a kernel; use the address
// returned by cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on `dev`, which must be the current device.
// Looked up on the first call per device and cached for the process lifetime:
// the address belongs to the device's primary context, so a cudaDeviceReset
// (which destroys that context and unloads this module) leaves the cached
// value stale; the public header tells callers not to use the entry point
// after one.
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int hs_solve_noalloc(hs_ctx* ctx, const double* alphas, int M, const double* thetas, int P, double* ufar,
                                void* stream) {
  if (!ctx) return HS_EINVAL;
  const int dev = hs::ctx_device(ctx);
  if (dev < 0 || dev >= kMaxDevices) return HS_EINVAL;
  if (cudaSetDevice(dev) != cudaSuccess) return HS_ECUDA;
  void* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess) return HS_ECUDA;
  return hs::solve_far_in_scratch(ctx, stream, alphas, M, thetas, P, ufar, base, kScratchBytes);
}
