// Jacobian by discrete reciprocity, misfit gradient and the Gauss-Newton
// normal equations.
//
// Theorem 3.1 gives a column of J as the far field of v with
//   Lap v + k^2 (1 - q) v = k^2 phi_m u_d.
// On the discrete system A x = b that is  J[(d,p), m] = l_p^T A^{-1} (k^2 phi_m u_d),
// so with the adjoint field z_p = A^{-T} l_p (the discrete counterpart of the
// adjoint field w of Theorem 3.2, computed by one transposed sweep of the
// stored merge operators per receiver) every entry is the contraction
//   J[(d,p), (m1,m2)] = k^2 sum_x z_p(x) u_d(x) s_m1(x1) s_m2(x2)
// over the interior collocation nodes: a Khatri-Rao product of forward and
// adjoint fields projected on the separable sine basis (eq. sineseries).
#include <algorithm>

#include "linalg.cuh"
#include "tree.cuh"

namespace hs {

// Interior rows of the leaf layout (r = (a-1)*14 + (b-1)) into the global
// interior grid G[j][gy][gx], gx = ix*14 + a-1, gy = iy*14 + b-1.
__global__ void k_leaf_to_grid(const double2* __restrict__ U, int rows, int nL, int nrhs, double2* __restrict__ G) {
  const int n14 = nL * 14;
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long tot = (long long)nL * nL * NI * nrhs;
  if (e >= tot) return;
  int j = (int)(e % nrhs);
  long long t = e / nrhs;
  int r = (int)(t % NI);
  int leaf = (int)(t / NI);
  int ix = leaf % nL, iy = leaf / nL;
  int a = r / 14, b = r % 14;
  G[((long long)j * n14 + iy * 14 + b) * n14 + ix * 14 + a] = U[((long long)leaf * rows + r) * nrhs + j];
}

void leaf_to_grid(cudaStream_t s, const double2* Uleaf, int nrows_leaf, int nL, int nrhs, double2* G) {
  long long tot = (long long)nL * nL * NI * nrhs;
  k_leaf_to_grid<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Uleaf, nrows_leaf, nL, nrhs, G);
  HS_COUNT_LAUNCH();
}

// Leaf layout (252 unknowns) into the natural node order out[j][leaf][a*16 + b]
// (corners, which are not unknowns, are 0).
__global__ void k_leaf_to_nodes(const double2* __restrict__ U, int nL, int nrhs, double2* __restrict__ out) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nleaf = nL * nL;
  long long tot = (long long)nleaf * 256 * nrhs;
  if (e >= tot) return;
  int node = (int)(e % 256);
  long long t = e / 256;
  int leaf = (int)(t % nleaf);
  int j = (int)(t / nleaf);
  int a = node / 16, b = node % 16;
  int r = -1;
  if (a >= 1 && a <= 14 && b >= 1 && b <= 14) r = (a - 1) * 14 + (b - 1);
  else if (b == 0 && a >= 1 && a <= 14) r = NI + a - 1;
  else if (a == 15 && b >= 1 && b <= 14) r = NI + 14 + b - 1;
  else if (b == 15 && a >= 1 && a <= 14) r = NI + 28 + a - 1;
  else if (a == 0 && b >= 1 && b <= 14) r = NI + 42 + b - 1;
  out[e] = r < 0 ? make_double2(0.0, 0.0) : U[((long long)leaf * NL + r) * nrhs + j];
}

void leaf_to_nodes(cudaStream_t s, const double2* Uleaf, int nL, int nrhs, double2* out) {
  long long tot = (long long)nL * nL * 256 * nrhs;
  k_leaf_to_nodes<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Uleaf, nL, nrhs, out);
  HS_COUNT_LAUNCH();
}

__global__ void k_int_sine(const double* __restrict__ xg, int n, int S, double* __restrict__ out) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int m = blockIdx.y + 1;
  if (g < n) out[(long long)(m - 1) * n + g] = sinpi(0.5 * m * (xg[g] + 1.0));
}

void interior_sine_tables(cudaStream_t s, const double* xg_int, int n, int S1, int S2, double* sx, double* sy) {
  k_int_sine<<<dim3((n + 127) / 128, S1), 128, 0, s>>>(xg_int, n, S1, sx);
  HS_COUNT_LAUNCH();
  k_int_sine<<<dim3((n + 127) / 128, S2), 128, 0, s>>>(xg_int, n, S2, sy);
  HS_COUNT_LAUNCH();
}

// Khatri-Rao rows of the contraction: W[c][g] = u_d(g) z_p(g) for the pairs
// c0 <= d*P + p < c0 + C over the interior grid points g (plane = nY * nX).
__global__ void k_khatri_rao(const double2* __restrict__ Ug, const double2* __restrict__ Zg, int P, long long plane,
                             long long c0, long long n, double2* __restrict__ W) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const long long c = c0 + e / plane, g = e % plane;
  const long long d = c / P, p = c % P;
  const double2 u = Ug[d * plane + g], z = Zg[p * plane + g];
  W[e] = make_double2(u.x * z.x - u.y * z.y, u.x * z.y + u.y * z.x);
}

// Scratch of the emulated products of a chunk of C pairs (the slices of its
// Khatri-Rao rows for the x-projection, then of its half-projected rows).
size_t contract_emulated_bytes(int C, int nX, int S1, int S2) {
  return oz_operand_bytes(S1, nX, 1, false) + oz_operand_bytes(S2, nX, 1, false) +
         std::max(oz_operand_bytes(2 * C * nX, nX, 1, true), oz_operand_bytes(2 * S1, nX, C, true));
}

int contract_chunk(int M, int P, int nX, int S1, size_t budget_bytes) {
  const size_t per = 16 * ((size_t)nX * nX + (size_t)nX * S1);
  long long c = (long long)(budget_bytes / per);
  // the second product is a batch of C launches' worth of grid.z; the emulated
  // x-projection has 2 nX / 128 row tiles per pair in grid.y
  long long cap = 32768;
  if (g_oz_enabled) cap = std::min<long long>(cap, 65535LL * 128 / (2LL * nX));
  return (int)std::max<long long>(1, std::min<long long>({c, (long long)M * P, cap}));
}

// Pairs per chunk of the FP32 contraction (8-byte W and T values): whole
// incidences (multiples of P) where the budget holds one, so that the
// Khatri-Rao tiles share each z_p read among several incidences.
int contract_chunk32(int M, int P, int nX, int S1, size_t budget_bytes) {
  const size_t per = 8 * ((size_t)nX * nX + (size_t)nX * S1);
  long long c = std::min<long long>({(long long)(budget_bytes / per), (long long)M * P, 32768});
  if (c >= P) c -= c % P;
  return (int)std::max<long long>(1, c);
}

// J[(d,p)][m1][m2] = k2 sum_gy sy[m2][gy] sum_gx sx[m1][gx] u_d[gy][gx] z_p[gy][gx],
// in chunks of C pairs: W = the pairs' Khatri-Rao rows (C x nY x nX), then
// T = W sx^T over gx (rows (pair, gy), one GEMM), then J_pair = T_pair^T sy^T
// over gy (a batch of S1 x S2 products).  W holds C*nX*nX and T C*nX*S1
// complex values.
// With the emulated FP64 product (g_oz_enabled) both projections run on the
// tensor cores: complex rows are read as pairs of real rows (re, im), and the
// sine tables are the transposed right operands; scratch (after T) holds the
// slices, contract_emulated_bytes(C, nX, S1, S2) bytes.
void contract_jacobian(cudaStream_t s, const double2* Ug, const double2* Zg, int M, int P, int nX, const double* sx,
                       const double* sy, int S1, int S2, double k2, double2* J, double2* W, double2* T, int C,
                       void* scratch, size_t scratch_bytes) {
  const long long plane = (long long)nX * nX, MP = (long long)M * P;
  const bool emu = g_oz_enabled && scratch && scratch_bytes >= contract_emulated_bytes(C, nX, S1, S2);
  char* base = reinterpret_cast<char*>(scratch);
  const size_t bsx = oz_operand_bytes(S1, nX, 1, false), bsy = oz_operand_bytes(S2, nX, 1, false);
  char *osx = base, *osy = base + bsx, *oa = base + bsx + bsy;
  if (emu) {  // the sine tables, sliced once as the right operands of both projections
    oz_slice(s, OzView{const_cast<double*>(sx), 0, nX, 0, 1, 1}, S1, nX, 1, false, osx);
    oz_slice(s, OzView{const_cast<double*>(sy), 0, nX, 0, 1, 1}, S2, nX, 1, false, osy);
  }
  for (long long c0 = 0; c0 < MP; c0 += C) {
    const int nc = (int)std::min<long long>(C, MP - c0);
    const long long n = nc * plane;
    bool done = false;
    if (emu) {
      double* Td = reinterpret_cast<double*>(T);
      double* Jd = reinterpret_cast<double*>(J + c0 * S1 * S2);
      // T[(pair, gy)][m1] = sum_gx (u_d z_p)[gy][gx] sx[m1][gx]: the Khatri-Rao rows are
      // sliced straight from the fields (no W)
      oz_slice_khatri_rao(s, Ug, Zg, P, nX, c0, nc, oa);
      const OzView vt{Td, 0, 2LL * S1, 1, 2, 2};
      done = oz_multiply(s, 2 * nc * nX, S1, nX, 1, 1.0, oa, osx, true, 0.0, vt) == cudaSuccess;
      // J_pair[m1][m2] = k2 sum_gy T_pair[gy][m1] sy[m2][gy]
      if (done) {
        const OzView vtt{Td, 2LL * nX * S1, 2, 1, 2LL * S1, 2}, vj{Jd, 2LL * S1 * S2, 2LL * S2, 1, 2, 2};
        oz_slice(s, vtt, 2 * S1, nX, nc, true, oa);
        done = oz_multiply(s, 2 * S1, S2, nX, nc, k2, oa, osy, true, 0.0, vj) == cudaSuccess;
      }
    }
    if (!done) {
      k_khatri_rao<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Ug, Zg, P, plane, c0, n, W);
      HS_COUNT_LAUNCH();
      gemm<double2, double, double2>(s, OP_N, OP_T, nc * nX, S1, nX, make_double2(1.0, 0.0), W, nX, 0, sx, nX, 0,
                                     make_double2(0.0, 0.0), T, S1, 0, 1);
      gemm<double2, double, double2>(s, OP_T, OP_T, S1, S2, nX, make_double2(k2, 0.0), T, S1, (long long)nX * S1, sy,
                                     nX, 0, make_double2(0.0, 0.0), J + c0 * S1 * S2, S2, (long long)S1 * S2, nc);
    }
  }
}

// Products with J without forming it, for iterative solves of the linearized
// problem: with the forward fields u_d and adjoint fields z_p on the interior
// grid (N = nX^2 points),
//   (J v)[d][p]  = sum_x z_p(x) (k2 u_d(x) q_v(x)),  q_v(x) = sum_m v_m s_m1(x1) s_m2(x2),
//   Re(J^H f)_m  = k2 sum_x s_m1(x1) s_m2(x2) Re sum_d u_d(x) sum_p conj(f_dp) z_p(x).
__global__ void k_weight_fields(const double2* __restrict__ Ug, const double* __restrict__ qv, double k2, long long N,
                                long long n, double2* __restrict__ Y) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double w = k2 * qv[e % N];
  const double2 u = Ug[e];
  Y[e] = make_double2(w * u.x, w * u.y);
}

__global__ void k_conj_copy(const double2* __restrict__ f, int n, double2* __restrict__ out) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = make_double2(f[e].x, -f[e].y);
}

// y = J v (M x P complex) for real v (S1 x S2); G1 (S2 x nX), qv (nX^2), Y (M x nX^2) scratch.
void apply_J(cudaStream_t s, const double2* Ug, const double2* Zg, int M, int P, int nX, const double* sx,
             const double* sy, int S1, int S2, double k2, const double* v, double* G1, double* qv, double2* Y,
             double2* y) {
  const long long N = (long long)nX * nX;
  // q_v[gy][gx] = sum_m2 sy[m2][gy] sum_m1 v[m1][m2] sx[m1][gx]
  gemm<double, double, double>(s, OP_T, OP_N, S2, nX, S1, 1.0, v, S2, 0, sx, nX, 0, 0.0, G1, nX, 0, 1);
  gemm<double, double, double>(s, OP_T, OP_N, nX, nX, S2, 1.0, sy, nX, 0, G1, nX, 0, 0.0, qv, nX, 0, 1);
  k_weight_fields<<<(unsigned)((N * M + 255) / 256), 256, 0, s>>>(Ug, qv, k2, N, N * M, Y);
  HS_COUNT_LAUNCH();
  gemm<double2, double2, double2>(s, OP_N, OP_T, M, P, (int)N, make_double2(1.0, 0.0), Y, (int)N, 0, Zg, (int)N, 0,
                                  make_double2(0.0, 0.0), y, P, 0, 1);
}

// g = Re(J^H f) (S1 x S2) for complex f (M x P); fc (M x P), Zmix (M x nX^2), h (nX^2), T1 (S1 x nX) scratch.
void apply_JH(cudaStream_t s, const double2* Ug, const double2* Zg, int M, int P, int nX, const double* sx,
              const double* sy, int S1, int S2, double k2, const double2* f, double2* fc, double2* Zmix, double* h,
              double* T1, double* g) {
  const long long N = (long long)nX * nX;
  k_conj_copy<<<(M * P + 255) / 256, 256, 0, s>>>(f, M * P, fc);
  HS_COUNT_LAUNCH();
  gemm<double2, double2, double2>(s, OP_N, OP_N, M, (int)N, P, make_double2(1.0, 0.0), fc, P, 0, Zg, (int)N, 0,
                                  make_double2(0.0, 0.0), Zmix, (int)N, 0, 1);
  gradient_combine(s, Ug, Zmix, M, N, h);
  gemm<double, double, double>(s, OP_N, OP_T, S1, nX, nX, 1.0, sx, nX, 0, h, nX, 0, 0.0, T1, nX, 0, 1);
  gemm<double, double, double>(s, OP_N, OP_T, S1, S2, nX, k2, T1, nX, 0, sy, nX, 0, 0.0, g, S2, 0, 1);
}

// Explicit complex FP32 Jacobian, for iterations that stop at a loose
// tolerance: the contraction of the FP32 Khatri-Rao rows with the real x-sine
// table (a complex-by-real FP32 product), then the batch of per-pair
// y-projections.
// LSQR then applies J32 and J32^H by the two products below, which read J32
// once each and accumulate in FP64, so that they stay exact transposes of one
// operator (products computed from the fields with independent FP32 rounding
// are not, and the bidiagonalisation amplifies that mismatch).
// W[c - c0][g] = u_d(g) z_p(g) for the pairs c = d P + p in [c0, c0 + nc):
// each thread takes one grid point g and a tile of KR_DT incidences x KR_PT
// receivers, so that every field value it reads serves several pairs (6
// bytes read per 8-byte output for whole tiles, against 16 when each pair
// reads its own z_p).  The products are taken in FP32 from the rounded
// factors: |u z| = |u| |z| for complex numbers, so each output stays within a
// few FP32 roundings of the exact product.
constexpr int KR_DT = 4, KR_PT = 8;
__device__ __forceinline__ float2 to_f2(double2 v) { return make_float2((float)v.x, (float)v.y); }

__global__ void k_khatri_rao32(const double2* __restrict__ Ug, const double2* __restrict__ Zg, int P,
                               long long plane, long long c0, int nc, int ptiles, float2* __restrict__ W) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= plane) return;
  const long long d0 = c0 / P + (long long)(blockIdx.y / ptiles) * KR_DT;
  const int p0 = (int)(blockIdx.y % ptiles) * KR_PT;
  const long long cend = c0 + nc;
  float2 z[KR_PT];
#pragma unroll
  for (int i = 0; i < KR_PT; ++i)
    z[i] = p0 + i < P ? to_f2(Zg[(long long)(p0 + i) * plane + g]) : make_float2(0.f, 0.f);
#pragma unroll
  for (int a = 0; a < KR_DT; ++a) {
    const long long cd = (d0 + a) * P;  // pair index of (d0 + a, 0)
    if (cd + p0 >= cend) break;         // pairs grow with d: the rest lie beyond the chunk
    if (cd + min(p0 + KR_PT, P) <= c0) continue;
    const float2 u = to_f2(Ug[(d0 + a) * plane + g]);
#pragma unroll
    for (int i = 0; i < KR_PT; ++i) {
      const long long c = cd + p0 + i;
      if (p0 + i < P && c >= c0 && c < cend)
        W[(c - c0) * plane + g] =
            make_float2(fmaf(u.x, z[i].x, -u.y * z[i].y), fmaf(u.x, z[i].y, u.y * z[i].x));
    }
  }
}

// sxr[g][m] = sx[m][g] and sy, both as FP32
__global__ void k_sine_tables32(const double* __restrict__ sx, const double* __restrict__ sy, int n, int S1, int S2,
                                float* __restrict__ sxr, float* __restrict__ sy32) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (long long)n * S1) sxr[e] = (float)sx[(e % S1) * n + e / S1];
  if (e < (long long)n * S2) sy32[e] = (float)sy[e];
}

void contract_jacobian32(cudaStream_t s, const double2* Ug, const double2* Zg, int M, int P, int nX, const double* sx,
                         const double* sy, int S1, int S2, double k2, float2* J, float2* sxc, float* sy32, float2* W,
                         float2* T, int C) {
  const long long plane = (long long)nX * nX, MP = (long long)M * P;
  const long long nt = (long long)nX * std::max(S1, S2);
  float* sxr = reinterpret_cast<float*>(sxc);  // the real x-sine table (half the buffer)
  k_sine_tables32<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(sx, sy, nX, S1, S2, sxr, sy32);
  HS_COUNT_LAUNCH();
  for (long long c0 = 0; c0 < MP; c0 += C) {
    const int nc = (int)std::min<long long>(C, MP - c0);
    const long long nd = (c0 + nc - 1) / P - c0 / P + 1;  // incidences the chunk meets
    const int ptiles = (P + KR_PT - 1) / KR_PT;
    k_khatri_rao32<<<dim3((unsigned)((plane + 255) / 256), (unsigned)((nd + KR_DT - 1) / KR_DT * ptiles)), 256, 0,
                     s>>>(Ug, Zg, P, plane, c0, nc, ptiles, W);
    HS_COUNT_LAUNCH();
    gemm<float2, float, float2>(s, OP_N, OP_N, nc * nX, S1, nX, make_float2(1.f, 0.f), W, nX, 0, sxr, S1, 0,
                                make_float2(0.f, 0.f), T, S1, 0, 1);
    gemm<float2, float, float2>(s, OP_T, OP_T, S1, S2, nX, make_float2((float)k2, 0.f), T, S1, (long long)nX * S1,
                                sy32, nX, 0, make_float2(0.f, 0.f), J + c0 * S1 * S2, S2, (long long)S1 * S2, nc);
  }
}

// Products with the FP32 Jacobian, in FP64 FMAs: LSQR needs J v and J^H u to
// be transposes of one operator to FP64 rounding (a mismatch of 1e-13, as
// double-FP32 sums leave, grew to 7e-4 in the iterate within 20 steps at
// k = 40).  GB300 issues FP64 at 1/64 of the FP32 rate and the FP32 -> FP64
// conversion runs on the same pipe, so the entries of J are widened in
// integer arithmetic instead: sign kept, exponent rebiased by 1023 - 127,
// mantissa shifted into place; subnormals normalised by their leading zeros;
// zero, infinities and NaN mapped to theirs.  Exact for every FP32 value.
__device__ __forceinline__ double f2d_int(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
  const int lz = __clz(m) - 8;  // subnormal: shifts that bring the leading 1 to bit 23
  unsigned long long ex, man = (unsigned long long)m << 29;
  if (e == 0) {
    ex = m ? (unsigned long long)(897 - lz) : 0ull;
    man = m ? (unsigned long long)((m << lz) & 0x7fffffu) << 29 : 0ull;
  } else {
    ex = e == 0xffu ? 0x7ffull : (unsigned long long)(e + 896);
  }
  return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) | (ex << 52) | man));
}

// y[r] = sum_m J[r][m] v[m] for complex FP32 J and real v: one warp per row,
// four elements in flight per lane.
__global__ void k_gemv32(const float2* __restrict__ J, const double* __restrict__ v, long long rows, int n,
                         double2* __restrict__ y) {
  const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  const float2* row = J + r * n;
  double ax = 0.0, ay = 0.0;
  int m = lane;
  for (; m + 96 < n; m += 128) {
    float2 a[4];
    double w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = row[m + 32 * i];
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i] = v[m + 32 * i];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      ax = fma(f2d_int(a[i].x), w[i], ax);
      ay = fma(f2d_int(a[i].y), w[i], ay);
    }
  }
  for (; m < n; m += 32) {
    const float2 a = row[m];
    const double w = v[m];
    ax = fma(f2d_int(a.x), w, ax);
    ay = fma(f2d_int(a.y), w, ay);
  }
  for (int o = 16; o > 0; o >>= 1) {
    ax += __shfl_down_sync(0xffffffffu, ax, o);
    ay += __shfl_down_sync(0xffffffffu, ay, o);
  }
  if (lane == 0) y[r] = make_double2(ax, ay);
}

// part[b][m] = sum over rows r of block b of Re(conj(J[r][m]) u[r]) for complex
// FP32 J: one column per thread, four rows in flight.
constexpr int kRowsPerPart = 256;
__global__ void __launch_bounds__(128) k_gemvT32(const float2* __restrict__ J, const double2* __restrict__ u,
                                                 long long rows, int n, double* __restrict__ part) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  const long long r0 = (long long)blockIdx.y * kRowsPerPart;
  const int nr = rows - r0 < kRowsPerPart ? (int)(rows - r0) : kRowsPerPart;
  const float2* col = J + r0 * n + m;
  const double2* ub = u + r0;
  double acc = 0.0;
  int i = 0;
  for (; i + 3 < nr; i += 4) {
    float2 a[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) a[t] = col[(long long)(i + t) * n];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const double2 w = ub[i + t];
      acc = fma(f2d_int(a[t].x), w.x, acc);
      acc = fma(f2d_int(a[t].y), w.y, acc);
    }
  }
  for (; i < nr; ++i) {
    const float2 a = col[(long long)i * n];
    const double2 w = ub[i];
    acc = fma(f2d_int(a.x), w.x, acc);
    acc = fma(f2d_int(a.y), w.y, acc);
  }
  part[(long long)blockIdx.y * n + m] = acc;
}

// The same two products on an FP64 Jacobian, in FP64: one warp per row for
// y = J v; part[b][m] as above.
__global__ void k_gemv64(const double2* __restrict__ J, const double* __restrict__ v, long long rows, int n,
                         double2* __restrict__ y) {
  const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  const double2* row = J + r * n;
  double ax = 0.0, ay = 0.0;
  for (int m = lane; m < n; m += 32) {
    const double2 a = row[m];
    const double w = v[m];
    ax = fma(a.x, w, ax);
    ay = fma(a.y, w, ay);
  }
  for (int o = 16; o > 0; o >>= 1) {
    ax += __shfl_down_sync(0xffffffffu, ax, o);
    ay += __shfl_down_sync(0xffffffffu, ay, o);
  }
  if (lane == 0) y[r] = make_double2(ax, ay);
}

__global__ void k_gemvT64(const double2* __restrict__ J, const double2* __restrict__ u, long long rows, int n,
                          double* __restrict__ part) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const long long r0 = (long long)blockIdx.y * kRowsPerPart;
  if (m >= n) return;
  const long long r1 = min(rows, r0 + kRowsPerPart);
  double acc = 0.0;
  for (long long r = r0; r < r1; ++r) {
    const double2 a = J[r * n + m];
    const double2 b = u[r];
    acc = fma(a.x, b.x, acc);
    acc = fma(a.y, b.y, acc);
  }
  part[(long long)blockIdx.y * n + m] = acc;
}

__global__ void k_sum_rows(const double* __restrict__ part, int nparts, int n, double* __restrict__ g) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  double acc = 0.0;
  for (int b = 0; b < nparts; ++b) acc += part[(long long)b * n + m];
  g[m] = acc;
}

int gemvT_parts(long long rows) { return (int)((rows + kRowsPerPart - 1) / kRowsPerPart); }

void gemv32(cudaStream_t s, const float2* J, long long rows, int n, const double* v, double2* y) {
  k_gemv32<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(J, v, rows, n, y);
  HS_COUNT_LAUNCH();
}
void gemvT32(cudaStream_t s, const float2* J, long long rows, int n, const double2* u, double* part, double* g) {
  const int np = gemvT_parts(rows);
  k_gemvT32<<<dim3((n + 127) / 128, np), 128, 0, s>>>(J, u, rows, n, part);
  HS_COUNT_LAUNCH();
  k_sum_rows<<<(n + 255) / 256, 256, 0, s>>>(part, np, n, g);
  HS_COUNT_LAUNCH();
}
void gemv64(cudaStream_t s, const double2* J, long long rows, int n, const double* v, double2* y) {
  k_gemv64<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(J, v, rows, n, y);
  HS_COUNT_LAUNCH();
}
void gemvT64(cudaStream_t s, const double2* J, long long rows, int n, const double2* u, double* part, double* g) {
  const int np = gemvT_parts(rows);
  k_gemvT64<<<dim3((n + 127) / 128, np), 128, 0, s>>>(J, u, rows, n, part);
  HS_COUNT_LAUNCH();
  k_sum_rows<<<(n + 255) / 256, 256, 0, s>>>(part, np, n, g);
  HS_COUNT_LAUNCH();
}

// Jst = [Re J; Im J] (2 rows x cols, real).
__global__ void k_split_stack(const double2* __restrict__ J, int rows, int cols, double* __restrict__ Jst) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  double2 v = J[e];
  Jst[e] = v.x;
  Jst[(long long)rows * cols + e] = v.y;
}

void split_stack(cudaStream_t s, const double2* J, int rows, int cols, double* Jst) {
  long long n = (long long)rows * cols;
  k_split_stack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(J, rows, cols, Jst);
  HS_COUNT_LAUNCH();
}

// JstT = [Re J; Im J]^T (cols x 2 rows) through 32 x 32 shared-memory tiles:
// reads along the columns of J, writes along the rows of JstT.
__global__ void k_split_stack_t(const double2* __restrict__ J, int rows, int cols, double* __restrict__ JstT) {
  __shared__ double2 t[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[i][threadIdx.x] = J[(long long)r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) {
      const double2 v = t[threadIdx.x][i];
      JstT[(long long)c * 2 * rows + r] = v.x;
      JstT[(long long)c * 2 * rows + rows + r] = v.y;
    }
  }
}

void split_stack_t(cudaStream_t s, const double2* J, int rows, int cols, double* JstT) {
  dim3 g((cols + 31) / 32, (rows + 31) / 32);
  k_split_stack_t<<<g, dim3(32, 8), 0, s>>>(J, rows, cols, JstT);
  HS_COUNT_LAUNCH();
}

size_t normal_matrix_emulated_bytes(int rows, int n) { return ozaki_scratch_bytes(n, n, rows, 1, false); }

// A = JstT JstT^T (n x n) for JstT (n x rows) by the emulated FP64 product.
bool normal_matrix_emulated(cudaStream_t s, double* JstT, int rows, int n, double* A, void* scratch, size_t bytes) {
  const OzView v{JstT, 0, rows, 0, 1, 1}, c{A, 0, n, 0, 1, 1};
  return ozaki_gemm(s, n, n, rows, 1, 1.0, v, v, true, 0.0, c, scratch, bytes) == cudaSuccess;
}

// A[r][c] = A[c][r] for the entries above the computed block-lower part
// (column block of c beyond the row block of r).
__global__ void k_mirror_upper(double* A, int n, int bs) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int r = (int)(e / n), c = (int)(e % n);
  if (c >= (r / bs + 1) * bs) A[e] = A[(long long)c * n + r];
}

// A = Jst^T Jst (n x n, symmetric) for Jst (rows x n): block rows of width bs,
// each the product with the columns up to and including its diagonal block,
// then the upper part mirrored (about (nb + 1) / (2 nb) of the full product's
// flops for nb blocks).
void normal_matrix(cudaStream_t s, const double* Jst, int rows, int n, double* A) {
  constexpr int bs = 256;
  if (n < 4 * bs) {
    gemm<double, double, double>(s, OP_T, OP_N, n, n, rows, 1.0, Jst, n, 0, Jst, n, 0, 0.0, A, n, 0, 1);
    return;
  }
  for (int r0 = 0; r0 < n; r0 += bs) {
    const int m = std::min(bs, n - r0), nc = std::min(n, r0 + bs);
    gemm<double, double, double>(s, OP_T, OP_N, m, nc, rows, 1.0, Jst + r0, n, 0, Jst, n, 0, 0.0,
                                 A + (long long)r0 * n, n, 0, 1);
  }
  const long long tot = (long long)n * n;
  k_mirror_upper<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(A, n, bs);
  HS_COUNT_LAUNCH();
}

// res = data - F; rst = [Re res; Im res]; out2 += sum |res|^2.
__global__ void k_residual(const double* __restrict__ data, const double2* __restrict__ F, int n,
                           double2* __restrict__ res, double* __restrict__ rst, double* __restrict__ out2) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (e < n) {
    double2 r = make_double2(data[2 * e] - F[e].x, data[2 * e + 1] - F[e].y);
    res[e] = r;
    if (rst) {
      rst[e] = r.x;
      rst[n + e] = r.y;
    }
    v = r.x * r.x + r.y * r.y;
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(out2, v);
}

void residual(cudaStream_t s, const double* data, const double2* F, int n, double2* res, double* rst, double* out2) {
  k_residual<<<(n + 255) / 256, 256, 0, s>>>(data, F, n, res, rst, out2);
  HS_COUNT_LAUNCH();
}

// A += lambda I with lambda = lambda_rel * trace(A) / n (one block).
__global__ void k_add_lambda(double* A, int n, double lambda_rel) {
  __shared__ double red[256];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += A[(long long)i * n + i];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  double lam = lambda_rel * red[0] / n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) A[(long long)i * n + i] += lam;
}

void add_lambda(cudaStream_t s, double* A, int n, double lambda_rel) {
  k_add_lambda<<<1, 256, 0, s>>>(A, n, lambda_rel);
  HS_COUNT_LAUNCH();
}

// hre[x] = Re sum_d Ug[d][x] Zmix[d][x].
__global__ void k_gradient_combine(const double2* __restrict__ Ug, const double2* __restrict__ Zmix, int M,
                                   long long npts, double* __restrict__ hre) {
  long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= npts) return;
  double v = 0.0;
  for (int d = 0; d < M; ++d) {
    double2 a = Ug[d * npts + x], b = Zmix[d * npts + x];
    v += a.x * b.x - a.y * b.y;
  }
  hre[x] = v;
}

void gradient_combine(cudaStream_t s, const double2* Ug, const double2* Zmix, int M, long long npts, double* hre) {
  k_gradient_combine<<<(unsigned)((npts + 255) / 256), 256, 0, s>>>(Ug, Zmix, M, npts, hre);
  HS_COUNT_LAUNCH();
}

// v <- -conj(v)
__global__ void k_conj_neg(double2* v, int n) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) v[e] = make_double2(-v[e].x, v[e].y);
}

void conj_neg(cudaStream_t s, double2* v, int n) {
  k_conj_neg<<<(n + 255) / 256, 256, 0, s>>>(v, n);
  HS_COUNT_LAUNCH();
}

__global__ void k_half(double* v) { v[0] *= 0.5; }

void half_in_place(cudaStream_t s, double* v) {
  k_half<<<1, 1, 0, s>>>(v);
  HS_COUNT_LAUNCH();
}

}  // namespace hs
