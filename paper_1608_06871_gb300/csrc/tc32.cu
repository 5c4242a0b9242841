// FP32 matrix products on the 5th-generation tensor cores by a three-term TF32
// split, for the dense contractions of the mixed-precision solver (leaf
// operators, merge products, the coupled root system, the sweeps).
//
// Every operand entry is split exactly x = hi + mid + lo with hi = tf32(x),
// mid = tf32(x - hi), lo = tf32(x - hi - mid) (round to nearest; 33 bits cover
// FP32's 24).  The tensor cores accumulate the six products whose weight is at
// least 2^-22 (hi hi, hi mid, mid hi, mid mid, hi lo, lo hi) in FP32; the three
// dropped ones are below 3 2^-33 of the product, so a product is as accurate
// as an FP32 one and the accumulation adds the usual FP32 rounding.  With two
// terms (hi hi + hi lo + lo hi, the common 3xTF32) each operand keeps only 22
// bits: the FP32 factors of the solver then contracted the refinement an order
// of magnitude less per pass (k = 70 needed a fourth pass), which cost more
// than the faster products saved.  A two-term FP16 split with power-of-two row
// scaling, at twice the TF32 rate, lost the low term of every entry more than
// 2^-17 below its row's largest (FP16's five exponent bits).
//
// Operand forms (real matrices A' m x k', B' n' x k', D' = A' B'^T):
//   complex A, complex B:  A' = A as floats (re, im interleaved along k, k' = 2k);
//                          B' rows 2j = (re, -im), 2j + 1 = (im, re) of column j
//                          at k' = 2l, 2l + 1: D' columns 2j, 2j + 1 = Re, Im C[:, j];
//   real A, complex B:     A' = A (k' = k); B' rows 2j, 2j + 1 = Re, Im of column j;
//   real A, real B:        A' = A, B' rows = columns of B.
// Split kernels write each operand once into three FP32 planes (hi, mid, lo;
// row-major, k' padded to a multiple of 4); the product kernel stages 32-wide
// k slices of the planes (128-byte rows) with TMA (three-dimensional maps
// {32 k', rows, 3 planes}, 128-byte swizzle, the MMA's K-major operand
// layout) into a ring of up to 216 KB: warp 0 loads, warp 1 issues the MMAs
// (M = 128, N = 64 or 128, K = 8; six per k step), warps 2..5 read the
// accumulator back.  Products with fewer output tiles than SMs split k over
// grid.z into FP32 partial planes, summed in order by a combine kernel.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <vector>

#include "linalg.cuh"

namespace hs {

bool prof_active(int family);
void prof_begin(cudaStream_t s, cudaEvent_t* a);
void prof_end(cudaStream_t s, cudaEvent_t a, double flops);

// Set to 1 by a split-TF32 product whose bounded mbarrier wait gave up (read
// and cleared by tc_timed_out with the other tensor-core flags).
__device__ int g_t32_timeout = 0;

namespace {

constexpr int TM_ = 128;        // A' rows per tile
constexpr int TKS = 32;         // k' per stage: one 128-byte row per operand row
constexpr int TTHREADS = 192;   // warp 0 TMA, warp 1 MMA, warps 2..5 epilogue
constexpr long long TWAIT = 1LL << 26;
constexpr int TRING = 216 * 1024;
constexpr int TPL = 3;          // planes per operand (hi, mid, lo)

template <int NT>
struct TCfg {
  static constexpr int A_PL = TM_ * 128;                    // one plane of the A tile (rows x 128 B)
  static constexpr int B_PL = NT * 128;
  static constexpr int STAGE = TPL * (A_PL + B_PL);
  static constexpr int ST = TRING / STAGE;                  // stages in the ring
  static constexpr int SMEM = ST * STAGE + 1024;
  // D = F32, A = B = TF32, both K-major, N = NT, M = 128
  static constexpr uint32_t IDESC =
      (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(TM_ >> 4) << 24);
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major, 128-byte swizzle (as TMA writes it): rows of 128 bytes, atoms of
// 8 rows (1024 bytes, the 8-row group stride); the k offset inside the row is
// added to the start address.
__device__ __forceinline__ uint64_t tdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ bool twait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < TWAIT; ++it) {
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

__device__ __forceinline__ void ttma3(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tld16(uint32_t ta, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(ta));
}

__device__ __forceinline__ float tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void split3(float x, float& hi, float& mid, float& lo) {
  hi = tf32(x);
  const float r = x - hi;  // exact
  mid = tf32(r);
  lo = tf32(r - mid);      // exact: r - mid has at most 13 significant bits
}

// Rows of a left operand: row r of batch b is src[b sb + r ld + 0 .. kk)
// (floats), written as the three planes over kp (zero beyond kk); four
// entries per thread, consecutive threads along the row.
__global__ void k_t32_split_rows(const float* __restrict__ src, long long ld, long long sb, int rows, int kk,
                                 long long total_rows, int kp, float* __restrict__ hi, long long plane) {
  const long long e4 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int q4 = kp / 4;
  if (e4 >= total_rows * q4) return;
  const long long w = e4 / q4;
  const int q = (int)(e4 % q4) * 4;
  const long long b = w / rows;
  const int r = (int)(w % rows);
  const float* x = src + b * sb + r * ld;
  float4 h, m, l;
  split3(q < kk ? x[q] : 0.f, h.x, m.x, l.x);
  split3(q + 1 < kk ? x[q + 1] : 0.f, h.y, m.y, l.y);
  split3(q + 2 < kk ? x[q + 2] : 0.f, h.z, m.z, l.z);
  split3(q + 3 < kk ? x[q + 3] : 0.f, h.w, m.w, l.w);
  *reinterpret_cast<float4*>(hi + w * kp + q) = h;
  *reinterpret_cast<float4*>(hi + plane + w * kp + q) = m;
  *reinterpret_cast<float4*>(hi + 2 * plane + w * kp + q) = l;
}

// Rows of B'^T from the columns of B through a shared-memory transpose: block
// = 32 columns x 64 rows of B (32 x 8 threads).  mode 2: complex A (rows
// 2j, 2j + 1 hold (re, -im), (im, re) at k' = 2l, 2l + 1); mode 1: real A (rows
// 2j, 2j + 1 = re, im at k' = l); mode 0: real B (row j at k' = l).
__global__ void k_t32_split_cols(const float* __restrict__ src, long long ld, long long sb, int k, int n, int mode,
                                 int kp, float* __restrict__ hi, long long plane) {
  __shared__ float2 tile[64][33];
  const int j0 = blockIdx.x * 32, l0 = blockIdx.y * 64, b = blockIdx.z;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const float* x = src + b * sb;
  const bool cplx = mode != 0;
  for (int q = ty; q < 64; q += 8) {
    const int l = l0 + q, j = j0 + tx;
    float2 v = make_float2(0.f, 0.f);
    if (l < k && j < n) v = cplx ? *reinterpret_cast<const float2*>(x + l * ld + 2 * j) : make_float2(x[l * ld + j], 0.f);
    tile[q][tx] = v;
  }
  __syncthreads();
  const int nrow = cplx ? 2 * n : n;
  // warp ty writes columns jj = ty, ty + 8, ..; its lanes run along l
  for (int jj = ty; jj < 32; jj += 8) {
    const int j = j0 + jj;
    if (j >= n) break;
    if (mode == 2) {
      const long long r0 = (long long)b * nrow + 2 * j;
      for (int q = tx; q < 64; q += 32) {
        const int kq = 2 * (l0 + q);
        if (kq >= kp) break;
        const float2 v = tile[q][jj];
        float a[3], c[3];
        split3(v.x, a[0], a[1], a[2]);
        split3(v.y, c[0], c[1], c[2]);
        // row 2j: (re, -im); row 2j + 1: (im, re)
#pragma unroll
        for (int t = 0; t < TPL; ++t) {
          *reinterpret_cast<float2*>(hi + t * plane + r0 * kp + kq) = make_float2(a[t], -c[t]);
          *reinterpret_cast<float2*>(hi + t * plane + (r0 + 1) * kp + kq) = make_float2(c[t], a[t]);
        }
      }
    } else {
      const long long r0 = (long long)b * nrow + (mode == 1 ? 2 * j : j);
      const int q = 2 * tx;  // two consecutive l per lane
      const int kq = l0 + q;
      if (kq < kp) {
        const float2 v0 = tile[q][jj], v1 = tile[q + 1][jj];
        float a0[3], a1[3];
        split3(v0.x, a0[0], a0[1], a0[2]);
        split3(v1.x, a1[0], a1[1], a1[2]);
#pragma unroll
        for (int t = 0; t < TPL; ++t)
          *reinterpret_cast<float2*>(hi + t * plane + r0 * kp + kq) = make_float2(a0[t], a1[t]);
        if (mode == 1) {
          float c0[3], c1[3];
          split3(v0.y, c0[0], c0[1], c0[2]);
          split3(v1.y, c1[0], c1[1], c1[2]);
#pragma unroll
          for (int t = 0; t < TPL; ++t)
            *reinterpret_cast<float2*>(hi + t * plane + (r0 + 1) * kp + kq) = make_float2(c0[t], c1[t]);
        }
      }
    }
  }
}

struct TParams {
  int m, n;          // output rows; output columns (complex columns when cplx)
  int nprime;        // rows of B' per batch item (columns of D')
  int stages;        // k' stages of the whole product
  int per_piece;     // stages per k piece (grid.z = batch * pieces)
  int pieces;
  int b_shared;
  int cplx;
  float2 alpha, beta;
  void* C;
  int ldc;
  long long sC;
  float* part;       // pieces > 1: partial planes [piece][batch][m][nprime]
};

template <int NT>
__global__ void __launch_bounds__(TTHREADS, 1)
    k_t32_mma(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TParams P) {
  using Cf = TCfg<NT>;
  constexpr int ST = Cf::ST;
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  __shared__ uint32_t tslot;
  __shared__ __align__(8) uint64_t full[ST], empty[ST], done;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.z / P.pieces, piece = blockIdx.z % P.pieces;
  const int tm = blockIdx.y, tn = blockIdx.x;
  const int rowA = b * P.m + tm * TM_;
  const int rowB = (P.b_shared ? 0 : b * P.nprime) + tn * NT;
  const int st0 = piece * P.per_piece;
  const int nst = min(P.per_piece, P.stages - st0);

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)), "r"(NT));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < ST; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&full[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&empty[i])), "r"(1));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&done)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      for (int i = 0; i < nst && ok; ++i) {
        const int st = i % ST;
        if (i >= ST) ok = twait(su32(&empty[st]), ((i / ST) - 1) & 1);
        if (!ok) break;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&full[st])), "r"(Cf::STAGE)
                     : "memory");
        const uint32_t base = su32(sm + st * Cf::STAGE);
        const int kx = (st0 + i) * TKS;
        ttma3(base, &mapA, kx, rowA, 0, su32(&full[st]));
        ttma3(base + TPL * Cf::A_PL, &mapB, kx, rowB, 0, su32(&full[st]));
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      for (int i = 0; i < nst && ok; ++i) {
        const int st = i % ST;
        ok = twait(su32(&full[st]), (i / ST) & 1);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t aB = su32(sm + st * Cf::STAGE), bB = aB + TPL * Cf::A_PL;
        // term pairs (a, b) of weight >= 2^-22, the small ones first
        constexpr int PA[6] = {1, 0, 2, 1, 0, 0}, PB[6] = {1, 2, 0, 0, 1, 0};
#pragma unroll
        for (int kh = 0; kh < TKS / 8; ++kh) {  // K = 8 TF32 (32 bytes) per MMA
#pragma unroll
          for (int t = 0; t < 6; ++t) {
            const uint64_t da = tdesc(aB + PA[t] * Cf::A_PL + kh * 32);
            const uint64_t db = tdesc(bB + PB[t] * Cf::B_PL + kh * 32);
            const uint32_t acc = (i > 0 || kh > 0 || t > 0) ? 1u : 0u;
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                "l"(da), "l"(db), "r"(Cf::IDESC), "r"(acc));
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            su32(&empty[st])));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&done)));
    }
  }
  const bool drained = twait(su32(&done), 0);
  ok = ok && drained;
  asm volatile("tcgen05.fence::after_thread_sync;");
  const bool all_ok = __syncthreads_and(ok ? 1 : 0) != 0;
  if (!all_ok && threadIdx.x == 0) atomicExch(&g_t32_timeout, 1);
  if (all_ok && warp >= 2) {
    const int quarter = warp & 3;
    const int r = tm * TM_ + quarter * 32 + lane;
    const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16);
    const bool row_ok = r < P.m;
    for (int c0 = 0; c0 < NT; c0 += 16) {
      uint32_t v[16];
      tld16(ta + (uint32_t)c0, v);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (!row_ok) continue;
      const int cb = tn * NT + c0;  // first column of D' in this chunk
      if (P.pieces > 1) {
        const long long nbatch = gridDim.z / P.pieces;
        float* out = P.part + (((long long)piece * nbatch + b) * P.m + r) * P.nprime;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int c = cb + q;
          if (c < P.nprime) out[c] = __uint_as_float(v[q]);
        }
      } else if (P.cplx) {
        float2* Cr = reinterpret_cast<float2*>(P.C) + b * P.sC + (long long)r * P.ldc;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int c = (cb >> 1) + q;
          if (c >= P.n) break;
          const float2 x = make_float2(__uint_as_float(v[2 * q]), __uint_as_float(v[2 * q + 1]));
          float2 o = make_float2(P.alpha.x * x.x - P.alpha.y * x.y, P.alpha.x * x.y + P.alpha.y * x.x);
          if (P.beta.x != 0.f || P.beta.y != 0.f) {
            const float2 y = Cr[c];
            o.x += P.beta.x * y.x - P.beta.y * y.y;
            o.y += P.beta.x * y.y + P.beta.y * y.x;
          }
          Cr[c] = o;
        }
      } else {
        float* Cr = reinterpret_cast<float*>(P.C) + b * P.sC + (long long)r * P.ldc;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int c = cb + q;
          if (c >= P.n) break;
          float o = P.alpha.x * __uint_as_float(v[q]);
          if (P.beta.x != 0.f) o += P.beta.x * Cr[c];
          Cr[c] = o;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NT));
}

// Sum of the k pieces (in piece order) into C with alpha and beta.
__global__ void k_t32_combine(const float* __restrict__ part, int pieces, int batch, int m, int n, int nprime,
                              int cplx, float2 alpha, float2 beta, void* C, int ldc, long long sC) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = (long long)batch * m * n;
  if (t >= tot) return;
  const int c = (int)(t % n);
  const long long br = t / n;  // b * m + r
  const int r = (int)(br % m);
  const long long b = br / m;
  const long long pstride = (long long)batch * m * nprime;
  const float* p = part + br * nprime;
  if (cplx) {
    float2 x = make_float2(0.f, 0.f);
    for (int q = 0; q < pieces; ++q) {
      x.x += p[q * pstride + 2 * c];
      x.y += p[q * pstride + 2 * c + 1];
    }
    float2* o = reinterpret_cast<float2*>(C) + b * sC + (long long)r * ldc + c;
    float2 y = make_float2(alpha.x * x.x - alpha.y * x.y, alpha.x * x.y + alpha.y * x.x);
    if (beta.x != 0.f || beta.y != 0.f) {
      const float2 z = *o;
      y.x += beta.x * z.x - beta.y * z.y;
      y.y += beta.x * z.y + beta.y * z.x;
    }
    *o = y;
  } else {
    float x = 0.f;
    for (int q = 0; q < pieces; ++q) x += p[q * pstride + c];
    float* o = reinterpret_cast<float*>(C) + b * sC + (long long)r * ldc + c;
    float y = alpha.x * x;
    if (beta.x != 0.f) y += beta.x * *o;
    *o = y;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_tenc = nullptr;
std::once_flag g_tenc_once;

bool tenc() {
  std::call_once(g_tenc_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_tenc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return g_tenc != nullptr;
}

// 3-D map over the planes [TPL][rows][kp] (FP32), box {32 k', box_rows, TPL}
// with the 128-byte swizzle of the MMA operand layout.
bool tmap(CUtensorMap* map, void* base, long long rows, int kp, int box_rows) {
  const cuuint64_t dims[3] = {(cuuint64_t)kp, (cuuint64_t)rows, TPL};
  const cuuint64_t strides[2] = {(cuuint64_t)kp * 4, (cuuint64_t)rows * kp * 4};
  const cuuint32_t box[3] = {(cuuint32_t)TKS, (cuuint32_t)box_rows, TPL};
  const cuuint32_t es[3] = {1, 1, 1};
  return g_tenc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline size_t al1k(size_t b) { return (b + 1023) & ~size_t(1023); }
inline long long cdiv(long long a, long long b) { return (a + b - 1) / b; }

// Scratch of the products, one buffer per (device, stream): products on one
// stream are ordered, so they can share it.  It only grows, and never while
// the stream is being captured (a captured product keeps its address; a grown
// buffer replaces it for later products and the old one is kept alive).
struct TScratch {
  void* p = nullptr;
  size_t bytes = 0;
};
std::mutex g_tmu;
std::map<std::pair<int, cudaStream_t>, TScratch> g_treg;
std::vector<void*> g_tretired;

void* t32_scratch(cudaStream_t s, size_t need) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_tmu);
  TScratch& sc = g_treg[{dev, s}];
  if (sc.bytes >= need) return sc.p;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
  const size_t want = std::max(need + need / 4, (size_t)64 << 20);
  void* p = nullptr;
  if (cudaMalloc(&p, want) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (sc.p) g_tretired.push_back(sc.p);
  sc.p = p;
  sc.bytes = want;
  return p;
}

template <int NT>
void set_attr() {
  static bool done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && done[dev]) return;
  cudaFuncSetAttribute(k_t32_mma<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, TCfg<NT>::SMEM);
  if (dev >= 0 && dev < 64) done[dev] = true;
}

template <int NT>
void launch_mma(cudaStream_t s, dim3 grid, const CUtensorMap& ma, const CUtensorMap& mb, const TParams& P) {
  set_attr<NT>();
  k_t32_mma<NT><<<grid, TTHREADS, TCfg<NT>::SMEM, s>>>(ma, mb, P);
  HS_COUNT_LAUNCH();
}

}  // namespace

bool t32_timed_out(cudaStream_t s) {
  int v = 0, z = 0;
  cudaStreamSynchronize(s);
  cudaMemcpyFromSymbolAsync(&v, g_t32_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (v) {
    cudaMemcpyToSymbolAsync(g_t32_timeout, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
  }
  return v != 0;
}

bool t32_gemm(cudaStream_t s, int mode, int m, int n, int k, float2 alpha, const float* A, long long lda,
              long long sA, const float* B, long long ldb, long long sB, float2 beta, void* C, int ldc, long long sC,
              int batch) {
  if (g_t32_mode == 0 || m <= 0 || n <= 0 || k <= 0 || batch <= 0 || batch > 65535 || !tenc()) return false;
  const bool cplx = mode != 0;
  const int kprime = mode == 2 ? 2 * k : k;
  const int nprime = cplx ? 2 * n : n;
  const int kp = (int)cdiv(kprime, 4) * 4;
  const bool b_shared = sB == 0 && batch > 1;
  const int nbB = b_shared ? 1 : batch;
  const int NT = nprime <= 64 ? 64 : 128;
  const long long tiles = cdiv(m, TM_) * cdiv(nprime, NT) * batch;
  const int stages = (int)cdiv(kp, TKS);
  // k pieces when the tiles leave SMs idle (one CTA per SM)
  int pieces = 1;
  if (tiles < 152 && stages >= 8) {
    pieces = (int)std::min<long long>(cdiv(152, tiles), stages / 4);
    pieces = std::max(1, std::min(pieces, 16));
    if ((long long)batch * pieces > 65535) pieces = 1;
  }
  const int per_piece = (int)cdiv(stages, pieces);
  pieces = (int)cdiv(stages, per_piece);
  const long long ra = (long long)batch * m, rb = (long long)nbB * nprime;
  const size_t pa = al1k((size_t)ra * kp * 4 * TPL), pb = al1k((size_t)rb * kp * 4 * TPL);
  const size_t pp = pieces > 1 ? al1k((size_t)pieces * batch * m * nprime * 4) : 0;
  char* base = static_cast<char*>(t32_scratch(s, pa + pb + pp));
  if (!base) return false;
  float* ta = reinterpret_cast<float*>(base);
  float* tb = reinterpret_cast<float*>(base + pa);
  float* part = pieces > 1 ? reinterpret_cast<float*>(base + pa + pb) : nullptr;
  CUtensorMap ma, mb;
  if (!tmap(&ma, ta, ra, kp, TM_) || !tmap(&mb, tb, rb, kp, NT)) return false;
  const bool prof = prof_active(3);
  cudaEvent_t ev = nullptr;
  if (prof) prof_begin(s, &ev);
  // operands
  k_t32_split_rows<<<(unsigned)cdiv(ra * (kp / 4), 256), 256, 0, s>>>(A, lda, sA, m, kprime, ra, kp, ta,
                                                                        (long long)ra * kp);
  HS_COUNT_LAUNCH();
  const int lrows = mode == 2 ? kp / 2 : kp;  // rows of B covered (with the zero tail)
  k_t32_split_cols<<<dim3((unsigned)cdiv(n, 32), (unsigned)cdiv(lrows, 64), nbB), dim3(32, 8), 0, s>>>(
      B, ldb, sB, k, n, mode, kp, tb, (long long)rb * kp);
  HS_COUNT_LAUNCH();
  TParams P;
  P.m = m;
  P.n = n;
  P.nprime = nprime;
  P.stages = stages;
  P.per_piece = per_piece;
  P.pieces = pieces;
  P.b_shared = b_shared ? 1 : 0;
  P.cplx = cplx ? 1 : 0;
  P.alpha = alpha;
  P.beta = beta;
  P.C = C;
  P.ldc = ldc;
  P.sC = sC;
  P.part = part;
  const dim3 grid((unsigned)cdiv(nprime, NT), (unsigned)cdiv(m, TM_), (unsigned)(batch * pieces));
  if (NT == 64) launch_mma<64>(s, grid, ma, mb, P);
  else launch_mma<128>(s, grid, ma, mb, P);
  if (pieces > 1) {
    const long long tot = (long long)batch * m * n;
    k_t32_combine<<<(unsigned)cdiv(tot, 256), 256, 0, s>>>(part, pieces, batch, m, n, nprime, cplx ? 1 : 0, alpha,
                                                           beta, C, ldc, sC);
    HS_COUNT_LAUNCH();
  }
  if (prof) prof_end(s, ev, (cplx ? (mode == 2 ? 8.0 : 4.0) : 2.0) * m * n * k * batch);
  return true;
}

}  // namespace hs
