// Status flags of the tensor-core kernels.  Every tcgen05 kernel bounds its
// mbarrier waits; one that gives up sets its translation unit's device flag
// (the split-TF32 product's in tc32.cu, the emulated-FP64 one's in ozaki.cu),
// and the library reads and clears them after the launches of an API call
// (HS_ETIMEOUT).  The flag defined here is the one a test raises from the host.
#include "linalg.cuh"

namespace hs {

// Raised from the host by the failure-injection hook (hs_raise_tc_timeout).
__device__ int g_tc_timeout = 0;

// Set the current device's timeout flag from the host (test hook: the next
// call that checks it reports HS_ETIMEOUT; no kernel waits on anything).
cudaError_t tc_raise_timeout_flag() {
  const int one = 1;
  return cudaMemcpyToSymbol(g_tc_timeout, &one, sizeof(int), 0, cudaMemcpyHostToDevice);
}

bool tc_timed_out(cudaStream_t s) {
  const bool others = oz_timed_out(s) || t32_timed_out(s);
  int v = 0, z = 0;
  cudaStreamSynchronize(s);
  cudaMemcpyFromSymbolAsync(&v, g_tc_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (v) {
    cudaMemcpyToSymbolAsync(g_tc_timeout, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
  }
  return v != 0 || others;
}

}  // namespace hs
