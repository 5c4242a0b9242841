// Complex FP32 GEMM on the 5th-generation tensor cores (tcgen05, TMEM).
//
// C = alpha A B + beta C for complex FP32 matrices (row-major, interleaved),
// used for the dense contractions of the mixed-precision solver (merge
// products, the coupled root system, the downward sweep).  FP32 accuracy is
// kept with the 3xTF32 split: every operand x = hi + lo with hi = tf32(x),
// lo = tf32(x - hi), and the product accumulates hi*hi + hi*lo + lo*hi in FP32
// in tensor memory.
//
// The complex product is a real product with twice the K and N:
//   A' = A as floats (m x 2k: re, im interleaved along k)
//   B' (2n rows x 2k, K-major): row j < n holds (re B[l][j], -im B[l][j]) at k' = 2l, 2l+1,
//                               row n + j holds (im B[l][j],  re B[l][j])
//   D' = A' B'^T = [Re C | Im C].
// Tile: 128 complex rows x 64 complex columns (D' is 128 x 128 FP32 in TMEM),
// K chunks of 16 complex (32 real) staged by all 128 threads into shared
// memory in the canonical K-major layout without swizzle (core matrices of 8
// rows x 16 bytes), two stages, with the next chunk prefetched into
// registers while the tensor cores work on the current one.  One thread
// issues the MMAs (M = 128, N = 128, K = 8) and commits them to an mbarrier.
#include <cstdint>

#include "linalg.cuh"

namespace hs {

// Set to 1 by a tensor-core GEMM whose bounded mbarrier wait gave up.
__device__ int g_tc_timeout = 0;

namespace {

constexpr int TM = 128;         // complex rows per tile
constexpr int TN = 64;          // complex columns per tile
constexpr int TKC = 16;         // complex k per chunk
constexpr int TK = 2 * TKC;     // real k per chunk (32)
constexpr int NR = 2 * TN;      // real output columns (128)
constexpr int TC_THREADS = 128;
constexpr int OP_BYTES = TM * TK * 4;            // one operand copy: 128 rows x 32 floats = 16 KB
constexpr int STAGE_BYTES = 4 * OP_BYTES;        // A hi, A lo, B' hi, B' lo
constexpr int TC_SMEM = 2 * STAGE_BYTES + 1024;  // two stages + alignment slack
constexpr uint32_t LBO = (TM / 8) * 128;         // bytes between core matrices along k (16 row groups)
constexpr uint32_t SBO = 128;                    // bytes between 8-row groups
// instruction descriptor: D = F32, A = B = TF32, both K-major, N = 128, M = 128
constexpr uint32_t IDESC =
    (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NR >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
constexpr long long WAIT_LIMIT = 1LL << 26;      // bounded mbarrier waits

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((LBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((SBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ float tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// float offset of element (row r, real k q) inside one operand copy
__device__ __forceinline__ int core_off(int r, int q) { return ((q >> 2) * (TM / 8) + (r >> 3)) * 32 + (r & 7) * 4 + (q & 3); }

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_cgemm_tc(int m, int n, int k, float2 alpha, const float2* __restrict__ A, int lda, long long sA,
               const float2* __restrict__ B, int ldb, long long sB, float2 beta, float2* __restrict__ C, int ldc,
               long long sC) {
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  __shared__ uint32_t tslot;
  __shared__ __align__(8) uint64_t mbar[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.z;
  A += b * sA;
  B += b * sB;
  C += b * sC;
  const int row0 = blockIdx.y * TM, col0 = blockIdx.x * TN;
  const int nchunk = (k + TKC - 1) / TKC;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)), "r"(NR));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&mbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;

  // register prefetch: A chunk 128 x 16 complex = 1024 float4 (8 per thread),
  // B chunk 16 x 64 complex = 512 float4 (4 per thread); a float4 is 2 complex
  float4 ra[8], rb[4];
  auto prefetch = [&](int ch) {
    const int kb = ch * TKC;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int q = tid + TC_THREADS * i;  // 0..1023
      int r = q >> 3, c2 = (q & 7) * 2;  // complex column pair within the chunk
      int gr = row0 + r, gk = kb + c2;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gr < m) {
        const float2* p = A + (long long)gr * lda + gk;
        if (gk < k) { v.x = p[0].x; v.y = p[0].y; }
        if (gk + 1 < k) { v.z = p[1].x; v.w = p[1].y; }
      }
      ra[i] = v;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int q = tid + TC_THREADS * i;  // 0..511
      int l = q >> 5, j2 = (q & 31) * 2;
      int gk = kb + l, gc = col0 + j2;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gk < k) {
        const float2* p = B + (long long)gk * ldb + gc;
        if (gc < n) { v.x = p[0].x; v.y = p[0].y; }
        if (gc + 1 < n) { v.z = p[1].x; v.w = p[1].y; }
      }
      rb[i] = v;
    }
  };
  auto stage_store = [&](int st) {
    float* Ahi = reinterpret_cast<float*>(sm + st * STAGE_BYTES);
    float* Alo = Ahi + OP_BYTES / 4;
    float* Bhi = Alo + OP_BYTES / 4;
    float* Blo = Bhi + OP_BYTES / 4;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int q = tid + TC_THREADS * i;
      int r = q >> 3, c4 = q & 7;  // real k' = 4 c4 .. 4 c4 + 3: one 16-byte core-matrix row
      float4 v = ra[i];
      float4 h = make_float4(tf32(v.x), tf32(v.y), tf32(v.z), tf32(v.w));
      float4 lo = make_float4(tf32(v.x - h.x), tf32(v.y - h.y), tf32(v.z - h.z), tf32(v.w - h.w));
      int off = core_off(r, 4 * c4);
      *reinterpret_cast<float4*>(Ahi + off) = h;
      *reinterpret_cast<float4*>(Alo + off) = lo;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int q = tid + TC_THREADS * i;
      int l = q >> 5, j2 = (q & 31) * 2;
      float4 v = rb[i];  // B[l][j2], B[l][j2+1]
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        float re = s ? v.z : v.x, im = s ? v.w : v.y;
        int j = j2 + s;
        // row j: (re, -im) at k' = 2l, 2l+1; row TN + j: (im, re)
        float e0 = re, e1 = -im, f0 = im, f1 = re;
        float h0 = tf32(e0), h1 = tf32(e1), g0 = tf32(f0), g1 = tf32(f1);
        int o1 = core_off(j, 2 * l), o2 = core_off(TN + j, 2 * l);
        Bhi[o1] = h0;
        Bhi[o1 + 1] = h1;
        Blo[o1] = tf32(e0 - h0);
        Blo[o1 + 1] = tf32(e1 - h1);
        Bhi[o2] = g0;
        Bhi[o2 + 1] = g1;
        Blo[o2] = tf32(f0 - g0);
        Blo[o2 + 1] = tf32(f1 - g1);
      }
    }
  };

  bool ok = true;
  prefetch(0);
  for (int ch = 0; ch < nchunk; ++ch) {
    const int st = ch & 1;
    if (ch >= 2) ok = ok && mbar_wait(su32(&mbar[st]), ((ch >> 1) - 1) & 1);  // MMAs of chunk ch-2 done
    stage_store(st);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      const uint32_t base = su32(sm + st * STAGE_BYTES);
      const uint32_t ahi = base, alo = base + OP_BYTES, bhi = base + 2 * OP_BYTES, blo = base + 3 * OP_BYTES;
#pragma unroll
      for (int ks = 0; ks < TK / 8; ++ks) {
        const uint32_t koff = ks * 2 * LBO;  // two core matrices of k per MMA
        const uint64_t dA[3] = {sdesc(ahi + koff), sdesc(ahi + koff), sdesc(alo + koff)};
        const uint64_t dB[3] = {sdesc(bhi + koff), sdesc(blo + koff), sdesc(bhi + koff)};
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          const uint32_t acc = (ch > 0 || ks > 0 || t > 0) ? 1u : 0u;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
              "l"(dA[t]), "l"(dB[t]), "r"(IDESC), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(&mbar[st])));
    }
    if (ch + 1 < nchunk) prefetch(ch + 1);
  }
  // wait for the last commit of each stage
  if (nchunk >= 1) ok = ok && mbar_wait(su32(&mbar[(nchunk - 1) & 1]), ((nchunk - 1) >> 1) & 1);
  if (nchunk >= 2) ok = ok && mbar_wait(su32(&mbar[(nchunk - 2) & 1]), ((nchunk - 2) >> 1) & 1);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!ok) atomicExch(&g_tc_timeout, 1);
  if (ok) {
    // epilogue: warp w owns TMEM lanes (= rows) 32 w .. 32 w + 31
    const int r = row0 + 32 * warp + lane;
    for (int c0 = 0; c0 < TN; c0 += 16) {
      uint32_t re[16], im[16];
      const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(re[0]), "=r"(re[1]), "=r"(re[2]), "=r"(re[3]), "=r"(re[4]), "=r"(re[5]), "=r"(re[6]), "=r"(re[7]),
            "=r"(re[8]), "=r"(re[9]), "=r"(re[10]), "=r"(re[11]), "=r"(re[12]), "=r"(re[13]), "=r"(re[14]),
            "=r"(re[15])
          : "r"(ta + c0));
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(im[0]), "=r"(im[1]), "=r"(im[2]), "=r"(im[3]), "=r"(im[4]), "=r"(im[5]), "=r"(im[6]), "=r"(im[7]),
            "=r"(im[8]), "=r"(im[9]), "=r"(im[10]), "=r"(im[11]), "=r"(im[12]), "=r"(im[13]), "=r"(im[14]),
            "=r"(im[15])
          : "r"(ta + TN + c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (r < m) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = col0 + c0 + j;
          if (c < n) {
            float2 d = make_float2(__uint_as_float(re[j]), __uint_as_float(im[j]));
            float2 v = alpha * d;
            float2* pc = C + (long long)r * ldc + c;
            if (!(beta.x == 0.f && beta.y == 0.f)) v = v + beta * (*pc);
            *pc = v;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NR));
}

}  // namespace

bool g_tc_enabled = true;  // process-wide switch (hs_set_tensor_cores)

bool cgemm_tc_eligible(int opA, int opB, int m, int n, int k, int batch) {
  return g_tc_enabled && opA == OP_N && opB == OP_N && m >= TM && n >= TN && k >= 4 * TKC && batch <= 65535;
}

void cgemm_tc(cudaStream_t s, int m, int n, int k, float2 alpha, const float2* A, int lda, long long sA,
              const float2* B, int ldb, long long sB, float2 beta, float2* C, int ldc, long long sC, int batch) {
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    cudaFuncSetAttribute(k_cgemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  dim3 grid((n + TN - 1) / TN, (m + TM - 1) / TM, batch);
  k_cgemm_tc<<<grid, TC_THREADS, TC_SMEM, s>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
  HS_COUNT_LAUNCH();
}

bool tc_timed_out(cudaStream_t s) {
  int v = 0, z = 0;
  cudaStreamSynchronize(s);
  cudaMemcpyFromSymbolAsync(&v, g_tc_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (v) {
    cudaMemcpyToSymbolAsync(g_tc_timeout, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
  }
  return v != 0;
}

}  // namespace hs
