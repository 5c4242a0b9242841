// FP64 matrix products on the 5th-generation tensor cores by exact integer
// slices (error-free splitting in the manner of Ozaki, Ogita, Oishi and Rump,
// 2012, with row / column scaling as in Ozaki, Uchino and Imamura's later
// variants), for the FP64 contractions of the Jacobian.
//
// C = alpha A B (+ beta C), A m x k and B k x n real FP64.  Every row i of A
// is scaled by 2^-ea_i so that its largest entry lies in [1/2, 1), every
// column j of B by 2^-eb_j, and the scaled values are split exactly into
// S = 8 slices of beta = 7 bits:
//   x 2^-e = sum_s a_s 2^(-7 (s + 1)) + tail,  a_0 in [-128, 128], a_s in [-64, 64],
// each an integer, hence exact in BF16.  The product of two slices is then an
// exact integer matrix; summed in FP32 it stays exact while every partial sum
// is an integer below 2^24.  The anti-diagonal d = s + t of the slice pairs
// (s + t <= 7: 36 pairs) carries the weight 2^(-7 (d + 2)), so the pairs of one
// diagonal accumulate into one FP32 accumulator in tensor memory:
//   |partial sum| <= K 4096 (d + 3) < 2^24  for K <= 384,
// which bounds the k extent of one launch (the host splits longer products
// and accumulates the pieces in FP64).  The epilogue recombines the 8 diagonal
// sums exactly in 64-bit integers (two groups of four, < 2^46 each) and rounds
// once to FP64.  What is dropped is the pairs with s + t >= 8, below
// 2^-55 k max|A_i.| max|B_.j| per entry, and one FP64 rounding per piece: the
// result stays within the FP64 product's own bound 2 k u |A| |B|.
//
// Kernel: one CTA per 128 x 64 output tile; warp 0 loads slice tiles with TMA
// (cp.async.bulk.tensor, three-dimensional maps over [slice][row][k], 32-wide
// k slices of 64-byte rows with the 64-byte swizzle) into a two-stage ring, warp 1 issues the tcgen05 BF16 MMAs (M = 128, N = 64 to 256,
// K = 16; 28 per stage of 32 k) into the eight diagonal accumulators (all
// 512 TMEM columns), warps 2..5 read them back.  Every mbarrier wait is
// bounded; a timeout sets the library's tensor-core timeout flag.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "linalg.cuh"

namespace hs {

bool prof_active(int family);
void prof_begin(cudaStream_t s, cudaEvent_t* a);
void prof_end(cudaStream_t s, cudaEvent_t a, double flops);

// Set to 1 by an emulated-FP64 product whose bounded mbarrier wait gave up
// (read and cleared by tc_timed_out with the tensor-core GEMM's own flag).
__device__ int g_oz_timeout = 0;

namespace {

constexpr int OZ_S = 8;          // slices per operand
constexpr int OZ_ND = 8;         // anti-diagonals kept (s + t <= 7)
constexpr int OZ_TM = 128;       // rows per tile
constexpr int OZ_TN = 64;        // columns per tile
constexpr int OZ_KS = 32;        // k per stage
constexpr int OZ_KMAX = 384;     // k per launch keeping every diagonal sum below 2^24 (a multiple of 32)
constexpr int OZ_THREADS = 192;  // warp 0 TMA, warp 1 MMA, warps 2..5 epilogue
constexpr int OZ_A_SL = OZ_TM * 2 * OZ_KS;  // one slice of the A tile: 128 rows x 64 bytes (8 KB)
constexpr int OZ_B_SL = OZ_TN * 2 * OZ_KS;  // same for B (4 KB)
constexpr int OZ_STAGE = OZ_S * (OZ_A_SL + OZ_B_SL);  // 96 KB
constexpr int OZ_SMEM = 2 * OZ_STAGE + 1024;
constexpr long long OZ_WAIT = 1LL << 26;
// instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t oz_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(OZ_TM >> 4) << 24);
}

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major, 64-byte swizzle (as TMA writes it): rows of 64 bytes (32 BF16),
// atoms of 8 rows (512 bytes, the 8-row group stride); the k offset inside the
// row is added to the start address.
__device__ __forceinline__ uint64_t oz_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

__device__ __forceinline__ bool oz_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < OZ_WAIT; ++it) {
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

__device__ __forceinline__ void oz_tma3(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void oz_ld16(uint32_t ta, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(ta));
}

// Element (b, i, k) of a strided FP64 view.
__device__ __forceinline__ long long vaddr(const OzView& v, long long b, long long i, long long k) {
  return b * v.sb + (i / v.ig) * v.si + (i % v.ig) * v.sg + k * v.sk;
}

// |x| as ordered 64-bit integers (the bit pattern of a non-negative double).
__device__ __forceinline__ long long abs_bits(double x) { return __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL; }

// round(x 2^(56 - e)) for |x| < 2^e, in integer arithmetic on the bit pattern
// (mantissa shifted by the exponent difference, rounded to nearest); 0 for
// zeros and subnormals, whose contribution is below the slices' resolution.
__device__ __forceinline__ long long fixed56(double x, int e) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0) return 0;
  const long long m = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;  // 53-bit significand
  const int sh = E - 1075 + 56 - e;                                     // x 2^(56-e) = m 2^sh, sh <= 3
  long long v;
  if (sh >= 0) v = m << sh;
  else if (sh > -60) v = (m + (1LL << (-sh - 1))) >> (-sh);
  else v = 0;
  return b < 0 ? -v : v;
}

// BF16 bits of a small integer |a| <= 2^8 (exact): the float from the magic
// constant 1.5 * 2^23 (so that negative a stay in its binade), whose upper 16
// bits are then the BF16 value.
__device__ __forceinline__ unsigned short small_bf16(int a) {
  const float f = __int_as_float(0x4B400000 + a) - 12582912.0f;
  return (unsigned short)(__float_as_uint(f) >> 16);
}

// The 8 balanced base-128 digits of a 56-bit fixed-point N (|N| < 2^56),
// written to o[s * plane]: N = H 2^28 + L with L in [-2^27, 2^27), then four
// digits from each 32-bit half (weights 2^21, 2^14, 2^7, 1 within it), each
// rounded to nearest: |a_0| <= 128, |a_s| <= 64 after, sum_s a_s 2^(49 - 7 s) = N.
__device__ __forceinline__ void put_digits(long long n, unsigned short* o, long long plane) {
  const long long hq = (n + (1LL << 27)) >> 28;
  int h = (int)hq, l = (int)(n - (hq << 28));
  int a;
  a = (h + (1 << 20)) >> 21; h -= a << 21; o[0] = small_bf16(a);
  a = (h + (1 << 13)) >> 14; h -= a << 14; o[plane] = small_bf16(a);
  a = (h + (1 << 6)) >> 7;   h -= a << 7;  o[2 * plane] = small_bf16(a);
  o[3 * plane] = small_bf16(h);
  a = (l + (1 << 20)) >> 21; l -= a << 21; o[4 * plane] = small_bf16(a);
  a = (l + (1 << 13)) >> 14; l -= a << 14; o[5 * plane] = small_bf16(a);
  a = (l + (1 << 6)) >> 7;   l -= a << 7;  o[6 * plane] = small_bf16(a);
  o[7 * plane] = small_bf16(l);
}

// Slices of the rows of a view (rows = A's rows, or B's columns): one warp
// per row, lanes along k; slices written to out[s][b * rpad + i][kk] (BF16,
// kpad wide, zero padded), the row's exponent to e[b * rpad + i].  Padding
// rows get zero slices.  All in integer arithmetic (the FP64 pipe is the
// scarce unit): the row's largest magnitude fixes e with max 2^-e in
// [1/2, 1); each entry becomes the 56-bit fixed-point integer
// N = round(x 2^(56 - e)), |N| < 2^56, whose balanced base-128 digits are the
// slices (put_digits), which represent N exactly.
__global__ void k_oz_slice(OzView v, int rows, int k, int rpad, int kpad, int batch, __nv_bfloat16* __restrict__ out,
                           int* __restrict__ e, int ldo, int col0) {
  const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long long total = (long long)batch * rpad;
  if (r >= total) return;
  const long long b = r / rpad;
  const int i = (int)(r % rpad);
  const long long plane = total * ldo;
  unsigned short* o = reinterpret_cast<unsigned short*>(out) + r * ldo + col0;
  const bool live = i < rows;
  // the row's piece (k <= OZ_KMAX) is read once into registers
  constexpr int KPL = OZ_KMAX / 32;
  double x[KPL];
  long long mx = 0;
#pragma unroll
  for (int q = 0; q < KPL; ++q) {
    const int kk = lane + 32 * q;
    x[q] = (live && kk < k) ? v.p[vaddr(v, b, i, kk)] : 0.0;
    mx = max(mx, abs_bits(x[q]));
  }
  for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  const int Emax = (int)(mx >> 52);
  const int ex = mx == 0 ? 0 : Emax - 1022;  // largest |x| in [2^(ex-1), 2^ex)
  if (lane == 0) e[r] = ex;
#pragma unroll
  for (int q = 0; q < KPL; ++q) {
    const int kk = lane + 32 * q;
    if (kk >= kpad) break;
    put_digits(fixed56(x[q], ex), o + kk, plane);
  }
}

// Slices of the Khatri-Rao rows of a chunk of (incidence, receiver) pairs, for
// the x-projection of the Jacobian: complex row (pair c, gy) of w = u_d z_p
// (d = (c0 + c) / P, p = (c0 + c) % P, fields on the interior grid,
// [rhs][gy][gx]) over gx in [k0, k0 + kc), split into its real part (row
// 2 (c nX + gy)) and imaginary part (row 2 (c nX + gy) + 1).  One warp per
// complex row; the product is formed in FP64 in registers and never stored.
__global__ void k_oz_slice_kr(const double2* __restrict__ Ug, const double2* __restrict__ Zg, int P, int nX,
                              long long c0, int nc, int k0, int kc, int rpad, int kpad, __nv_bfloat16* __restrict__ out,
                              int* __restrict__ e) {
  const long long r2 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r2 >= (long long)nc * nX) return;
  const long long c = c0 + r2 / nX, gy = r2 % nX, plane = (long long)nX * nX;
  const double2* u = Ug + (c / P) * plane + gy * nX + k0;
  const double2* z = Zg + (c % P) * plane + gy * nX + k0;
  constexpr int KPL = OZ_KMAX / 32;
  double wr[KPL], wi[KPL];
  long long mr = 0, mi = 0;
#pragma unroll
  for (int q = 0; q < KPL; ++q) {
    const int kk = lane + 32 * q;
    double2 w = make_double2(0.0, 0.0);
    if (kk < kc) {
      const double2 a = u[kk], b = z[kk];
      w = make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
    }
    wr[q] = w.x;
    wi[q] = w.y;
    mr = max(mr, abs_bits(w.x));
    mi = max(mi, abs_bits(w.y));
  }
  for (int off = 16; off > 0; off >>= 1) {
    mr = max(mr, __shfl_xor_sync(0xffffffffu, mr, off));
    mi = max(mi, __shfl_xor_sync(0xffffffffu, mi, off));
  }
  const int er = mr == 0 ? 0 : (int)(mr >> 52) - 1022, ei = mi == 0 ? 0 : (int)(mi >> 52) - 1022;
  const long long plane_s = (long long)rpad * kpad;
  unsigned short* o_re = reinterpret_cast<unsigned short*>(out) + (2 * r2) * kpad;
  unsigned short* o_im = o_re + kpad;
  if (lane == 0) {
    e[2 * r2] = er;
    e[2 * r2 + 1] = ei;
  }
#pragma unroll
  for (int q = 0; q < KPL; ++q) {
    const int kk = lane + 32 * q;
    if (kk >= kpad) break;
    put_digits(fixed56(wr[q], er), o_re + kk, plane_s);
    put_digits(fixed56(wi[q], ei), o_im + kk, plane_s);
  }
}

// Zero slices of the padding rows [first, rpad) of every slice plane.
__global__ void k_oz_zero_rows(long long first, int rpad, int kpad, __nv_bfloat16* __restrict__ out, int* __restrict__ e) {
  const long long n = (long long)(rpad - first) * kpad;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * OZ_S) return;
  const int s = (int)(t / n);
  const long long j = t % n;
  out[(long long)s * rpad * kpad + first * kpad + j] = __float2bfloat16_rn(0.f);
  if (s == 0 && j % kpad == 0) e[first + j / kpad] = 0;
}

struct OzParams {
  int m, n, k, mpad, npad, kpad, nb_batch_b;  // nb_batch_b: 0 when B is shared by every batch
  // zpieces: grid.z runs over the pieces of k (pl wide, k the whole extent) of one
  // product instead of over a batch; piece z writes its own output plane z
  int zpieces, pl;
  double alpha, beta;
  const int* ea;
  const int* eb;
  OzView C;
};

__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_mma(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, OzParams P) {
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  __shared__ uint32_t tslot;
  __shared__ __align__(8) uint64_t full[2], empty[2], done;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.z;  // batch, or piece of k
  const int tm = blockIdx.y, tn = blockIdx.x;
  const bool zp = P.zpieces != 0;
  const int rowA = (zp ? 0 : b * P.mpad) + tm * OZ_TM;
  const int rowB = (zp ? 0 : (P.nb_batch_b ? b : 0) * P.npad) + tn * OZ_TN;
  const int kbase = zp ? b * P.pl : 0;
  const int nst = zp ? (min(P.pl, P.k - kbase) + OZ_KS - 1) / OZ_KS : P.kpad / OZ_KS;
  const int bB = zp ? b : (P.nb_batch_b ? b : 0);  // exponent plane of B

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
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
        const int st = i & 1;
        if (i >= 2) ok = oz_wait(su32(&empty[st]), ((i >> 1) - 1) & 1);
        if (!ok) break;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&full[st])), "r"(OZ_STAGE)
                     : "memory");
        const uint32_t base = su32(sm + st * OZ_STAGE);
        const int kx = kbase + i * OZ_KS;
        oz_tma3(base, &mapA, kx, rowA, 0, su32(&full[st]));
        oz_tma3(base + OZ_S * OZ_A_SL, &mapB, kx, rowB, 0, su32(&full[st]));
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      for (int i = 0; i < nst && ok; ++i) {
        const int st = i & 1;
        ok = oz_wait(su32(&full[st]), (i >> 1) & 1);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t aB = su32(sm + st * OZ_STAGE), bB = aB + OZ_S * OZ_A_SL;
        // The B slices of a k block lie back to back (slice t at rows 64 t .. 64 t + 63)
        // and the diagonal accumulators are adjacent in TMEM (diagonal d at columns
        // 64 d ..), so one MMA with N = 64 w multiplies A_s by B_t .. B_(t+w-1) into
        // diagonals s + t .. s + t + w - 1: per slice s the 8 - s pairs take
        // MMAs of N = 256, 128 and 64 (14 per 16 k instead of 36).
#pragma unroll 1
        for (int kh = 0; kh < OZ_KS / 16; ++kh) {
#pragma unroll 1
          for (int s = 0; s < OZ_S; ++s) {
            const uint64_t da = oz_desc(aB + s * OZ_A_SL + kh * 32);
            const uint32_t acc = (i > 0 || kh > 0 || s > 0) ? 1u : 0u;
            int t = 0;
#pragma unroll 1
            while (t + s < OZ_ND) {
              const int left = OZ_ND - s - t;
              const int w = left >= 4 ? 4 : left >= 2 ? 2 : 1;
              const uint64_t db = oz_desc(bB + t * OZ_B_SL + kh * 32);
              const uint32_t idesc = oz_idesc(w * OZ_TN);
              asm volatile(
                  "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem + (uint32_t)((s + t) * OZ_TN)),
                  "l"(da), "l"(db), "r"(idesc), "r"(acc));
              t += w;
            }
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            su32(&empty[st])));
      }
      // one more commit tracks every MMA issued above
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&done)));
    }
  }
  // everyone: wait until the tensor cores are done with TMEM and the stages
  const bool drained = oz_wait(su32(&done), 0);
  ok = ok && drained;
  asm volatile("tcgen05.fence::after_thread_sync;");
  const bool all_ok = __syncthreads_and(ok ? 1 : 0) != 0;
  if (!all_ok && threadIdx.x == 0) atomicExch(&g_oz_timeout, 1);
  if (all_ok && warp >= 2) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = tile rows; lane = row
    const int quarter = warp & 3;
    const int r = tm * OZ_TM + quarter * 32 + lane;
    const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16);
    const bool row_ok = r < P.m;
    const int ea = row_ok ? P.ea[(long long)b * P.mpad + r] : 0;
    for (int c0 = 0; c0 < OZ_TN; c0 += 16) {
      long long hi[16], lo[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) hi[j] = lo[j] = 0;
#pragma unroll 1
      for (int d = 0; d < OZ_ND; ++d) {
        uint32_t v[16];
        oz_ld16(ta + (uint32_t)(d * OZ_TN + c0), v);
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const long long x = (long long)__float2int_rn(__uint_as_float(v[j]));  // an exact integer
          if (d < 4)
            hi[j] = hi[j] * 128 + x;  // 2^7: one slice width
          else
            lo[j] = lo[j] * 128 + x;
        }
      }
      if (row_ok) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = tn * OZ_TN + c0 + j;
          if (c >= P.n) continue;
          // sum_d C_d 2^(-7 (d + 2)) = hi 2^-35 + lo 2^-63, then the row and column scales
          const double val = fma((double)lo[j], 0x1p-63, (double)hi[j] * 0x1p-35);
          const int eb = P.eb[(long long)bB * P.npad + c];
          double* pc = P.C.p + vaddr(P.C, b, r, c);
          const double out = P.alpha * scalbn(val, ea + eb);
          *pc = P.beta == 0.0 ? out : fma(P.beta, *pc, out);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool encode_fn() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return g_encode != nullptr;
}

// 3-D map over slices [OZ_S][rows][kpad] (BF16), box {32 k, box_rows, all
// slices} with the 64-byte swizzle of the MMA operand layout.
bool make_map(CUtensorMap* map, void* base, long long rows, int kpad, int box_rows) {
  const cuuint64_t dims[3] = {(cuuint64_t)kpad, (cuuint64_t)rows, (cuuint64_t)OZ_S};
  const cuuint64_t strides[2] = {(cuuint64_t)kpad * 2, (cuuint64_t)rows * kpad * 2};
  const cuuint32_t box[3] = {(cuuint32_t)OZ_KS, (cuuint32_t)box_rows, (cuuint32_t)OZ_S};
  const cuuint32_t es[3] = {1, 1, 1};
  return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline long long rup(long long x, long long m) { return (x + m - 1) / m * m; }

}  // namespace

bool g_oz_enabled = true;  // process-wide switch (hs_set_fp64_emulation)

bool oz_timed_out(cudaStream_t s) {
  int v = 0, z = 0;
  cudaStreamSynchronize(s);
  cudaMemcpyFromSymbolAsync(&v, g_oz_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (v) {
    cudaMemcpyToSymbolAsync(g_oz_timeout, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
  }
  return v != 0;
}

size_t ozaki_scratch_bytes(int m, int n, int k, int batch, bool b_shared) {
  const long long kp = rup(std::min(k, OZ_KMAX), OZ_KS), mp = rup(m, OZ_TM), np = rup(n, OZ_TN);
  const long long nbB = b_shared ? 1 : batch;
  const size_t a = ((size_t)OZ_S * batch * mp * kp * 2 + 1023) / 1024 * 1024 + ((size_t)batch * mp * 4 + 1023) / 1024 * 1024;
  const size_t b = ((size_t)OZ_S * nbB * np * kp * 2 + 1023) / 1024 * 1024 + ((size_t)nbB * np * 4 + 1023) / 1024 * 1024;
  return a + b;
}

namespace {

void set_smem_attr() {
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    cudaFuncSetAttribute(k_oz_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
}

// One launch of the tile kernel over a piece of k: sliced operands sa / sbt
// (rows padded to mp / np, kp wide) and their exponents.
cudaError_t launch_piece(cudaStream_t s, int m, int n, int kc, long long kp, long long mp, long long np, int batch,
                         bool b_shared, double alpha, double beta, __nv_bfloat16* sa, const int* ea,
                         __nv_bfloat16* sbt, const int* eb, OzView C) {
  CUtensorMap ma, mb;
  const long long ra = batch * mp, rb = (b_shared ? 1 : batch) * np;
  if (!make_map(&ma, sa, ra, (int)kp, OZ_TM) || !make_map(&mb, sbt, rb, (int)kp, OZ_TN)) return cudaErrorInvalidValue;
  OzParams P;
  P.m = m;
  P.n = n;
  P.k = kc;
  P.mpad = (int)mp;
  P.npad = (int)np;
  P.kpad = (int)kp;
  P.nb_batch_b = b_shared ? 0 : 1;
  P.zpieces = 0;
  P.pl = 0;
  P.alpha = alpha;
  P.beta = beta;
  P.ea = ea;
  P.eb = eb;
  P.C = C;
  dim3 grid((unsigned)(np / OZ_TN), (unsigned)(mp / OZ_TM), (unsigned)batch);
  const bool prof = prof_active(4);
  cudaEvent_t ev = nullptr;
  if (prof) prof_begin(s, &ev);
  k_oz_mma<<<grid, OZ_THREADS, OZ_SMEM, s>>>(ma, mb, P);
  HS_COUNT_LAUNCH();
  if (prof) prof_end(s, ev, 2.0 * m * n * kc * batch);  // FP64-equivalent flops
  return cudaSuccess;
}

size_t align_up(size_t b) { return (b + 1023) & ~size_t(1023); }

// Length of the pieces k is cut into: as equal as possible, at most OZ_KMAX,
// a multiple of the stage depth (the last piece takes the rest).
int piece_len(int k) {
  const int np = (k + OZ_KMAX - 1) / OZ_KMAX;
  return (int)std::min<long long>(OZ_KMAX, rup((k + np - 1) / np, OZ_KS));
}

// Byte layout of a sliced operand: piece after piece, each the slices
// [OZ_S][batch * rpad][kp] and the exponents [batch * rpad].
struct Piece {
  size_t slices, exps, next;
  long long kp;
  int kc;
};
Piece piece_at(size_t off, int k0, int k, long long rows_total) {
  Piece p;
  p.kc = std::min(piece_len(k), k - k0);
  p.kp = rup(p.kc, OZ_KS);
  p.slices = off;
  p.exps = off + align_up((size_t)OZ_S * rows_total * p.kp * 2);
  p.next = p.exps + align_up((size_t)rows_total * 4);
  return p;
}

}  // namespace

size_t oz_operand_bytes(int rows, int k, int batch, bool is_a) {
  const long long rt = (long long)batch * rup(rows, is_a ? OZ_TM : OZ_TN);
  size_t off = 0;
  for (int k0 = 0; k0 < k; k0 += piece_len(k)) off = piece_at(off, k0, k, rt).next;
  return off;
}

void oz_slice(cudaStream_t s, OzView v, int rows, int k, int batch, bool is_a, void* buf) {
  const long long rpad = rup(rows, is_a ? OZ_TM : OZ_TN), rt = batch * rpad;
  char* base = reinterpret_cast<char*>(buf);
  size_t off = 0;
  for (int k0 = 0; k0 < k; k0 += piece_len(k)) {
    const Piece p = piece_at(off, k0, k, rt);
    OzView w = v;
    w.p += k0 * v.sk;
    k_oz_slice<<<(unsigned)((rt + 7) / 8), 256, 0, s>>>(w, rows, p.kc, (int)rpad, (int)p.kp, batch,
                                                      reinterpret_cast<__nv_bfloat16*>(base + p.slices),
                                                      reinterpret_cast<int*>(base + p.exps), (int)p.kp, 0);
    HS_COUNT_LAUNCH();
    off = p.next;
  }
}

void oz_slice_khatri_rao(cudaStream_t s, const double2* Ug, const double2* Zg, int P, int nX, long long c0, int nc,
                         void* buf) {
  const int rows = 2 * nc * nX;
  const long long rpad = rup(rows, OZ_TM);
  char* base = reinterpret_cast<char*>(buf);
  size_t off = 0;
  for (int k0 = 0; k0 < nX; k0 += piece_len(nX)) {
    const Piece p = piece_at(off, k0, nX, rpad);
    __nv_bfloat16* sl = reinterpret_cast<__nv_bfloat16*>(base + p.slices);
    int* ex = reinterpret_cast<int*>(base + p.exps);
    const long long warps = (long long)nc * nX;
    k_oz_slice_kr<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(Ug, Zg, P, nX, c0, nc, k0, p.kc, (int)rpad, (int)p.kp,
                                                             sl, ex);
    HS_COUNT_LAUNCH();
    if (rpad > rows) {
      const long long n = (rpad - rows) * p.kp * OZ_S;
      k_oz_zero_rows<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rows, (int)rpad, (int)p.kp, sl, ex);
      HS_COUNT_LAUNCH();
    }
    off = p.next;
  }
}

cudaError_t oz_multiply(cudaStream_t s, int m, int n, int k, int batch, double alpha, const void* Aop, const void* Bop,
                        bool b_shared, double beta, OzView C) {
  if (m <= 0 || n <= 0 || k <= 0 || batch <= 0 || batch > 65535) return cudaErrorInvalidValue;
  if (!encode_fn()) return cudaErrorNotSupported;
  set_smem_attr();
  const long long mp = rup(m, OZ_TM), np = rup(n, OZ_TN);
  char* a = const_cast<char*>(reinterpret_cast<const char*>(Aop));
  char* b = const_cast<char*>(reinterpret_cast<const char*>(Bop));
  size_t oa = 0, ob = 0;
  for (int k0 = 0; k0 < k; k0 += piece_len(k)) {
    const Piece pa = piece_at(oa, k0, k, batch * mp), pb = piece_at(ob, k0, k, (b_shared ? 1 : batch) * np);
    const cudaError_t e =
        launch_piece(s, m, n, pa.kc, pa.kp, mp, np, batch, b_shared, alpha, k0 == 0 ? beta : 1.0,
                     reinterpret_cast<__nv_bfloat16*>(a + pa.slices), reinterpret_cast<const int*>(a + pa.exps),
                     reinterpret_cast<__nv_bfloat16*>(b + pb.slices), reinterpret_cast<const int*>(b + pb.exps), C);
    if (e != cudaSuccess) return e;
    oa = pa.next;
    ob = pb.next;
  }
  return cudaGetLastError();
}

// ---- split-k products: one launch per real product, pieces of k along grid.z ----

namespace {
// C = alpha sum_p (P0 - P1) + i alpha sum_p (P2 + P3) (+ beta C), pieces summed in order.
__global__ void k_oz_zcombine(const double* __restrict__ P0, const double* __restrict__ P1,
                              const double* __restrict__ P2, const double* __restrict__ P3, int npc, int m, int n,
                              double alpha, double beta, double2* __restrict__ C, int ldc) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long mn = (long long)m * n;
  if (e >= mn) return;
  double re = 0.0, im = 0.0;
  for (int p = 0; p < npc; ++p) {
    re += P0[p * mn + e] - P1[p * mn + e];
    im += P2[p * mn + e] + P3[p * mn + e];
  }
  double2* c = C + (e / n) * ldc + (e % n);
  const double2 v = make_double2(alpha * re, alpha * im);
  *c = beta == 0.0 ? v : make_double2(v.x + beta * c->x, v.y + beta * c->y);
}

int npieces(int k) { return (k + piece_len(k) - 1) / piece_len(k); }
}  // namespace

size_t oz_wide_bytes(int rows, int k, bool is_a) {
  const long long rpad = rup(rows, is_a ? OZ_TM : OZ_TN), kt = (long long)npieces(k) * piece_len(k);
  return align_up((size_t)OZ_S * rpad * kt * 2) + align_up((size_t)npieces(k) * rpad * 4);
}

size_t oz_partial_bytes(int m, int n, int k) { return align_up((size_t)npieces(k) * m * n * 8); }

void oz_slice_wide(cudaStream_t s, OzView v, int rows, int k, bool is_a, void* buf) {
  const long long rpad = rup(rows, is_a ? OZ_TM : OZ_TN);
  const int pl = piece_len(k), kt = npieces(k) * pl;
  char* base = reinterpret_cast<char*>(buf);
  __nv_bfloat16* sl = reinterpret_cast<__nv_bfloat16*>(base);
  int* ex = reinterpret_cast<int*>(base + align_up((size_t)OZ_S * rpad * kt * 2));
  for (int p = 0, k0 = 0; k0 < k; ++p, k0 += pl) {
    const int kc = std::min(pl, k - k0);
    OzView w = v;
    w.p += k0 * v.sk;
    k_oz_slice<<<(unsigned)((rpad + 7) / 8), 256, 0, s>>>(w, rows, kc, (int)rpad, (int)rup(kc, OZ_KS), 1, sl,
                                                        ex + (long long)p * rpad, kt, k0);
    HS_COUNT_LAUNCH();
  }
}

cudaError_t oz_multiply_wide(cudaStream_t s, int m, int n, int k, const void* Aop, const void* Bop, double* partial) {
  if (m <= 0 || n <= 0 || k <= 0) return cudaErrorInvalidValue;
  if (!encode_fn()) return cudaErrorNotSupported;
  set_smem_attr();
  const long long mp = rup(m, OZ_TM), np = rup(n, OZ_TN);
  const int pl = piece_len(k), npc = npieces(k), kt = npc * pl;
  char* a = const_cast<char*>(reinterpret_cast<const char*>(Aop));
  char* b = const_cast<char*>(reinterpret_cast<const char*>(Bop));
  CUtensorMap ma, mb;
  if (!make_map(&ma, a, mp, kt, OZ_TM) || !make_map(&mb, b, np, kt, OZ_TN)) return cudaErrorInvalidValue;
  OzParams P;
  P.m = m;
  P.n = n;
  P.k = k;
  P.mpad = (int)mp;
  P.npad = (int)np;
  P.kpad = kt;
  P.nb_batch_b = 1;
  P.zpieces = 1;
  P.pl = pl;
  P.alpha = 1.0;
  P.beta = 0.0;
  P.ea = reinterpret_cast<const int*>(a + align_up((size_t)OZ_S * mp * kt * 2));
  P.eb = reinterpret_cast<const int*>(b + align_up((size_t)OZ_S * np * kt * 2));
  P.C = OzView{partial, (long long)m * n, n, 0, 1, 1};
  dim3 grid((unsigned)(np / OZ_TN), (unsigned)(mp / OZ_TM), (unsigned)npc);
  const bool prof = prof_active(4);
  cudaEvent_t ev = nullptr;
  if (prof) prof_begin(s, &ev);
  k_oz_mma<<<grid, OZ_THREADS, OZ_SMEM, s>>>(ma, mb, P);
  HS_COUNT_LAUNCH();
  if (prof) prof_end(s, ev, 2.0 * m * n * k);
  return cudaGetLastError();
}

cudaError_t oz_zmul_wide(cudaStream_t s, int m, int n, int k, const void* Are, const void* Aim, const void* Bre,
                         const void* Bim, double alpha, double beta, double2* C, int ldc, void* partials) {
  const size_t pb = oz_partial_bytes(m, n, k);
  double* P[4];
  for (int i = 0; i < 4; ++i) P[i] = reinterpret_cast<double*>(reinterpret_cast<char*>(partials) + i * pb);
  cudaError_t e = oz_multiply_wide(s, m, n, k, Are, Bre, P[0]);
  if (e == cudaSuccess) e = oz_multiply_wide(s, m, n, k, Aim, Bim, P[1]);
  if (e == cudaSuccess) e = oz_multiply_wide(s, m, n, k, Are, Bim, P[2]);
  if (e == cudaSuccess) e = oz_multiply_wide(s, m, n, k, Aim, Bre, P[3]);
  if (e != cudaSuccess) return e;
  const long long mn = (long long)m * n;
  k_oz_zcombine<<<(unsigned)((mn + 255) / 256), 256, 0, s>>>(P[0], P[1], P[2], P[3], npieces(k), m, n, alpha, beta,
                                                             C, ldc);
  HS_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t ozaki_gemm(cudaStream_t s, int m, int n, int k, int batch, double alpha, OzView A, OzView Bt, bool b_shared,
                       double beta, OzView C, void* scratch, size_t scratch_bytes) {
  if (m <= 0 || n <= 0 || k <= 0 || batch <= 0 || batch > 65535) return cudaErrorInvalidValue;
  if (!encode_fn()) return cudaErrorNotSupported;
  if (ozaki_scratch_bytes(m, n, k, batch, b_shared) > scratch_bytes) return cudaErrorInvalidValue;
  set_smem_attr();
  const long long mp = rup(m, OZ_TM), np = rup(n, OZ_TN);
  const long long nbB = b_shared ? 1 : batch;
  // piece by piece, slicing each piece of both operands into the same scratch
  for (int k0 = 0; k0 < k; k0 += piece_len(k)) {
    const Piece pa = piece_at(0, k0, k, batch * mp), pb = piece_at(pa.next, k0, k, nbB * np);
    char* base = reinterpret_cast<char*>(scratch);
    OzView a = A, bt = Bt;
    a.p += k0 * A.sk;
    bt.p += k0 * Bt.sk;
    const long long ra = batch * mp, rb = nbB * np;
    k_oz_slice<<<(unsigned)((ra + 7) / 8), 256, 0, s>>>(a, m, pa.kc, (int)mp, (int)pa.kp, batch,
                                                      reinterpret_cast<__nv_bfloat16*>(base + pa.slices),
                                                      reinterpret_cast<int*>(base + pa.exps), (int)pa.kp, 0);
    HS_COUNT_LAUNCH();
    k_oz_slice<<<(unsigned)((rb + 7) / 8), 256, 0, s>>>(bt, n, pb.kc, (int)np, (int)pb.kp, (int)nbB,
                                                      reinterpret_cast<__nv_bfloat16*>(base + pb.slices),
                                                      reinterpret_cast<int*>(base + pb.exps), (int)pb.kp, 0);
    HS_COUNT_LAUNCH();
    const cudaError_t e =
        launch_piece(s, m, n, pa.kc, pa.kp, mp, np, batch, b_shared, alpha, k0 == 0 ? beta : 1.0,
                     reinterpret_cast<__nv_bfloat16*>(base + pa.slices), reinterpret_cast<const int*>(base + pa.exps),
                     reinterpret_cast<__nv_bfloat16*>(base + pb.slices), reinterpret_cast<const int*>(base + pb.exps),
                     C);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace hs
