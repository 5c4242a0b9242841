// LU panel factorisation (columns [j0, j0 + nb) of a batch of n x n matrices)
// for the blocked right-looking LU of linalg.cu.
//
// Short panels (at most PR = 256 rows below j0) are factored with partial
// pivoting inside shared memory by one CTA per matrix, one thread per row: a
// block argmax per column, the row swap, the scaling and the rank-1 update
// all touch shared memory only.  The same row permutation is then applied to
// the columns outside the panel through a shared-memory staging buffer.
//
// Tall panels (the 1792-row coupled root system, the top merge levels) use
// tournament pivoting: sets of up to 256 rows are factored independently with
// partial pivoting (one CTA each) and each keeps its nb pivot rows; the
// candidates of 8 sets form the next round's sets until one set remains, whose
// partial-pivoting order gives the panel's pivot rows.  Those rows are swapped
// to the top (LAPACK swap sequence in piv) with their factored nb x nb block
// from the final round (partial pivoting inside the pivot rows reproduces that
// order), and the multipliers below solve L21 U11 = A21.  The sets of a round are
// independent, so the per-column latency of the pivot search is paid on 256
// rows in shared memory instead of on the whole column in global memory.
//
// Scratch for the candidate lists lives in piv[j0 + nb .. n) of each matrix,
// which later panels overwrite: for m = n - j0 > 256 rows it needs
// ceil(m / 256) nb + ... + 1 + 4 nb ints, below m - nb for nb = 32.
#include <algorithm>
#include <climits>
#include <mutex>
#include <utility>
#include <vector>

#include "linalg.cuh"

namespace hs {
namespace {

constexpr int PR = 256;      // rows per shared-memory tile (one thread per row)
constexpr int PNB = 32;      // panel width of the blocked LU
constexpr int PT = 256;      // threads of the tile kernels
constexpr int APPLY_CH = 32;  // columns per CTA of the row-permutation kernel

// Magnitude used for pivot selection, in the panel's own precision.
template <typename E> struct pmag;
template <> struct pmag<double> { using T = double; __device__ static double of(double a) { return fabs(a); } };
template <> struct pmag<double2> { using T = double; __device__ static double of(double2 a) { return a.x * a.x + a.y * a.y; } };
template <> struct pmag<float> { using T = float; __device__ static float of(float a) { return fabsf(a); } };
template <> struct pmag<float2> { using T = float; __device__ static float of(float2 a) { return a.x * a.x + a.y * a.y; } };

// 1 / x with one correctly rounded reciprocal: real x directly; complex x as
// conj(x) / |x|^2, or, where |x|^2 could leave the normal range, x = 2^e (a + i b)
// with the power of two from the larger component's exponent (exact), then
// (a - i b) / (a^2 + b^2) 2^-e.  The multipliers are formed as x_i (1 / pivot),
// as LAPACK's unblocked LU does.
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float2 recip(float2 x) {
  const float n2 = fmaf(x.x, x.x, x.y * x.y);
  if (n2 > 1e-30f && n2 < 1e30f) {  // |x|^2 safely inside the normal range
    const float d = __frcp_rn(n2);
    return make_float2(x.x * d, -x.y * d);
  }
  const int e = ilogbf(fmaxf(fabsf(x.x), fabsf(x.y)));
  const float a = scalbnf(x.x, -e), b = scalbnf(x.y, -e);
  const float d = scalbnf(__frcp_rn(fmaf(a, a, b * b)), -e);
  return make_float2(a * d, -b * d);
}
__device__ __forceinline__ double2 recip(double2 x) {
  const double n2 = fma(x.x, x.x, x.y * x.y);
  if (n2 > 1e-290 && n2 < 1e290) {
    const double d = __drcp_rn(n2);
    return make_double2(x.x * d, -x.y * d);
  }
  const int e = ilogb(fmax(fabs(x.x), fabs(x.y)));
  const double a = scalbn(x.x, -e), b = scalbn(x.y, -e);
  const double d = scalbn(__drcp_rn(fma(a, a, b * b)), -e);
  return make_double2(a * d, -b * d);
}

// Factor the rows x nb tile T (row stride ld, shared memory) with partial
// pivoting, one thread per row (blockDim.x = PT >= rows).  The rows stay where
// they are: each thread tracks the logical position of its own row (mylg), a
// pivot step only relabels two rows, and the thread whose row became a pivot
// row stops updating it, so every other thread can read the pivot row in
// place.  Per column there is a single barrier, after the warps publish their
// candidates (magnitude, then lowest logical position, as LAPACK's first
// maximum; FP32 magnitudes are reduced with redux.sync on their bit
// patterns).  The column loop is not unrolled (a small instruction footprint:
// the per-column latency is the point here); the thread keeps its row in
// registers and mirrors every updated entry to the tile.
// On return, loc[r] is the tile row holding logical row r, rid[] is permuted
// into logical order, sp[j] (if not NULL) receives the logical row swapped
// with row j at step j, and *zc is lowered to the first column whose pivot is
// exactly zero (that column is then left unscaled).
template <typename E>
__device__ void tile_lu(E* T, int ld, int rows, int nb, int* rid, int* loc, int* sp, int* zc) {
  using M = typename pmag<E>::T;
  constexpr int NW = PT / 32;
  __shared__ M wbest[2][NW];
  __shared__ int wkey[2][NW];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int steps = min(rows, nb);
  bool active = t < rows;
  int mylg = t;
  const int myid = active ? rid[t] : 0;
  E* row = T + t * ld;
  // the thread's row in registers (entries right of the current column are
  // the live ones); shared memory holds a mirror that the others read when
  // this row becomes the pivot row
  E r[PNB];
#pragma unroll
  for (int c = 0; c < PNB; ++c) r[c] = (active && c < nb) ? row[c] : el<E>::zero();
  for (int j = 0; j < steps; ++j) {
    const int pb = j & 1;
    M best = active ? pmag<E>::of(row[j]) : M(-1);
    int key = active ? (mylg << 8) | t : INT_MAX;  // logical position, then tile row
    if constexpr (sizeof(M) == 4) {
      // FP32 magnitudes: the warp maximum of their bit patterns (ordered for
      // non-negative floats; +1 keeps an active zero above an inactive row),
      // then the smallest key among the lanes holding it: two redux.sync
      unsigned mb = active ? __float_as_uint(best) + 1u : 0u;
      mb = __reduce_max_sync(0xffffffffu, mb);
      key = (int)__reduce_min_sync(0xffffffffu, (active && __float_as_uint(best) + 1u == mb) ? (unsigned)key
                                                                                            : 0xffffffffu);
      if (lane == 0) { wbest[pb][warp] = __uint_as_float(mb); wkey[pb][warp] = key; }
      __syncthreads();
      const unsigned wb = lane < NW ? __float_as_uint(wbest[pb][lane]) : 0u;
      const unsigned wk = lane < NW ? (unsigned)wkey[pb][lane] : 0xffffffffu;
      const unsigned bb = __reduce_max_sync(0xffffffffu, wb);
      key = (int)__reduce_min_sync(0xffffffffu, wb == bb ? wk : 0xffffffffu);
    } else {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const M ob = __shfl_down_sync(0xffffffffu, best, o);
        const int ok = __shfl_down_sync(0xffffffffu, key, o);
        if (ob > best || (ob == best && ok < key)) { best = ob; key = ok; }
      }
      if (lane == 0) { wbest[pb][warp] = best; wkey[pb][warp] = key; }
      __syncthreads();
      best = wbest[pb][0];
      key = wkey[pb][0];
#pragma unroll
      for (int w = 1; w < NW; ++w) {
        const M ob = wbest[pb][w];
        const int ok = wkey[pb][w];
        if (ob > best || (ob == best && ok < key)) { best = ob; key = ok; }
      }
    }
    const int p = key & 255, lp = key >> 8;
    if (sp && t == 0) sp[j] = lp;
    if (t == p) {
      active = false;
      mylg = j;
    } else if (mylg == j) {
      mylg = lp;
    }
    const E* prow = T + p * ld;
    const E pv = prow[j];
    if (!(pmag<E>::of(pv) > M(0))) {
      if (t == 0) atomicMin(zc, j);
    } else if (active) {
      const E l = row[j] * recip(pv);
      row[j] = l;
      // rank-1 update in registers, in groups of eight columns (groups left of
      // the column are skipped, warp-uniformly); each group's pivot entries are
      // loaded before its mirror stores are issued
#pragma unroll
      for (int g = 0; g < PNB / 8; ++g) {
        if (8 * g + 7 > j) {
          E u[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) u[q] = 8 * g + q < nb ? prow[8 * g + q] : el<E>::zero();
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int c = 8 * g + q;
            if (c > j && c < nb) {
              r[c] = fmsc(r[c], l, u[q]);
              row[c] = r[c];
            }
          }
        }
      }
    }
  }
  __syncthreads();
  if (t < rows) {
    loc[mylg] = t;
    rid[mylg] = myid;
  }
  __syncthreads();
}

// Stage rows x nb elements into the tile T (row stride ld): tile row r is
// source row ids[r] (or row0 + r without ids) of A (row stride lda).  One warp
// per row, lanes along the columns, eight rows in flight per warp.
template <typename E>
__device__ void load_rows(E* T, int ld, int rows, int nb, const E* A, int lda, const int* ids, int row0) {
  constexpr int NW = PT / 32, RF = 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r0 = warp * RF; r0 < rows; r0 += NW * RF) {
    E v[RF];
#pragma unroll
    for (int q = 0; q < RF; ++q) {
      const int r = r0 + q;
      v[q] = (r < rows && lane < nb) ? A[(long long)(ids ? ids[r] : row0 + r) * lda + lane] : el<E>::zero();
    }
#pragma unroll
    for (int q = 0; q < RF; ++q)
      if (r0 + q < rows && lane < nb) T[(r0 + q) * ld + lane] = v[q];
  }
}

// Short panel (m = n - j0 <= PR rows): one CTA per matrix.
template <typename E>
__global__ void __launch_bounds__(PT) k_panel_small(E* A, int lda, long long sA, int n, int j0, int nb, int* piv,
                                                    long long sP, int* info) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E* T = reinterpret_cast<E*>(smem_raw);
  __shared__ int rid[PR], loc[PR];
  __shared__ int sp[PNB];
  __shared__ int aff_d[2 * PNB], aff_s[2 * PNB];
  __shared__ int zc, naff;
  const int b = blockIdx.x, t = threadIdx.x;
  A += b * sA;
  piv += b * sP;
  const int m = n - j0, ld = nb + 1;
  load_rows<E>(T, ld, m, nb, A + j0, lda, nullptr, j0);
  if (t < m) rid[t] = t;
  if (t == 0) zc = INT_MAX;
  __syncthreads();
  tile_lu<E>(T, ld, m, nb, rid, loc, sp, &zc);
  for (int e = t; e < m * nb; e += PT) {
    const int r = e / nb, c = e % nb;
    A[(long long)(j0 + r) * lda + j0 + c] = T[loc[r] * ld + c];
  }
  if (t == 0) {
    const int steps = min(m, nb);
    for (int j = 0; j < steps; ++j) piv[j0 + j] = j0 + sp[j];
    if (zc != INT_MAX && info[b] == 0) info[b] = j0 + zc + 1;
    int k = 0;  // rows whose content changed: row r now holds old row rid[r]
    for (int r = 0; r < m && k < 2 * PNB; ++r)
      if (rid[r] != r) { aff_d[k] = r; aff_s[k] = rid[r]; ++k; }
    naff = k;
  }
  __syncthreads();
  // same permutation on the columns outside the panel, staged through T
  const int na = naff, cols_out = n - nb;
  for (int c0 = 0; c0 < cols_out && na > 0; c0 += APPLY_CH) {
    for (int e = t; e < na * APPLY_CH; e += PT) {
      const int a = e / APPLY_CH, cc = c0 + e % APPLY_CH;
      if (cc < cols_out) T[e] = A[(long long)(j0 + aff_s[a]) * lda + (cc < j0 ? cc : cc + nb)];
    }
    __syncthreads();
    for (int e = t; e < na * APPLY_CH; e += PT) {
      const int a = e / APPLY_CH, cc = c0 + e % APPLY_CH;
      if (cc < cols_out) A[(long long)(j0 + aff_d[a]) * lda + (cc < j0 ? cc : cc + nb)] = T[e];
    }
    __syncthreads();
  }
}

// One tournament round: set blockIdx.x of matrix blockIdx.y.  Round 0 takes
// rows j0 + 256 s .. ; later rounds take up to 256 candidate rows from the
// previous round's list (entries < 0 are empty).  Writes the set's nb pivot
// rows (absolute row numbers, in pivot order) to out, or, in the final round
// (one set), the factored pivot block, the LAPACK swap sequence
// piv[j0 .. j0 + nb) and the list of rows to move.
template <typename E>
__global__ void __launch_bounds__(PT) k_tp_select(E* A, int lda, long long sA, int n, int j0, int nb, int* piv,
                                                  long long sP, int* info, int in_off, int nin, int out_off,
                                                  int final_round, int aff_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E* T = reinterpret_cast<E*>(smem_raw);
  __shared__ int rid[PR], loc[PR];
  __shared__ int wsum[PT / 32];
  __shared__ int zc;
  __shared__ int kpos[2 * PNB], korig[2 * PNB];
  const int b = blockIdx.y, set = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  A += b * sA;
  piv += b * sP;
  int* W = piv + j0 + nb;  // scratch: rows of later panels' pivots
  int myrow = -1;
  if (in_off < 0) {
    const int r = j0 + set * PR + t;
    if (r < n) myrow = r;
  } else {
    const int e = set * PR + t;
    if (e < nin) myrow = W[in_off + e];
  }
  // compact the valid rows, in order (ballot prefix sums)
  const unsigned bal = __ballot_sync(0xffffffffu, myrow >= 0);
  if (lane == 0) wsum[warp] = __popc(bal);
  if (t == 0) zc = INT_MAX;
  __syncthreads();
  int off = 0, rows = 0;
  for (int w = 0; w < PT / 32; ++w) {
    if (w < warp) off += wsum[w];
    rows += wsum[w];
  }
  if (myrow >= 0) rid[off + __popc(bal & ((1u << lane) - 1u))] = myrow;
  __syncthreads();
  const int ld = nb + 1;
  load_rows<E>(T, ld, rows, nb, A + j0, lda, rid, 0);
  __syncthreads();
  tile_lu<E>(T, ld, rows, nb, rid, loc, nullptr, &zc);
  if (!final_round) {
    if (t < nb) W[out_off + set * nb + t] = t < rows ? rid[t] : -1;
    return;
  }
  // the top nb rows of T are the factored pivot block (L11 \ U11): store it
  // in the pivot rows' panel columns, which the row moves carry to j0 .. j0 + nb
  for (int e = t; e < nb * nb; e += PT) {
    const int r = e / nb, c = e % nb;
    A[(long long)rid[r] * lda + j0 + c] = T[loc[r] * ld + c];
  }
  if (t == 0) {
    if (zc != INT_MAX && info[b] == 0) info[b] = j0 + zc + 1;
    // LAPACK swap sequence bringing rid[0 .. nb) to rows j0 .. j0 + nb, and
    // the resulting moves (kpos[k] now holds original row korig[k])
    int np = 0;
    const int steps = min(rows, nb);
    for (int j = 0; j < steps; ++j) {
      const int target = j0 + j, pj = rid[j];
      int q = pj;
      for (int k = 0; k < np; ++k)
        if (korig[k] == pj) { q = kpos[k]; break; }
      piv[j0 + j] = q;
      if (q != target) {
        int it = -1, iq = -1, vt = target;
        for (int k = 0; k < np; ++k) {
          if (kpos[k] == target) { it = k; vt = korig[k]; }
          if (kpos[k] == q) iq = k;
        }
        if (it < 0) { kpos[np] = target; it = np++; }
        korig[it] = pj;
        if (iq < 0) { kpos[np] = q; iq = np++; }
        korig[iq] = vt;
      }
    }
    int k2 = 0;
    int* aff = W + aff_off;
    for (int k = 0; k < np; ++k)
      if (korig[k] != kpos[k]) {
        aff[1 + k2] = kpos[k];
        aff[1 + 2 * PNB + k2] = korig[k];
        ++k2;
      }
    aff[0] = k2;
  }
}

// Move the rows listed by the final round (all n columns), through shared memory.
template <typename E>
__global__ void __launch_bounds__(PT) k_tp_apply(E* A, int lda, long long sA, int n, const int* piv, long long sP,
                                                 int aff_at) {
  __shared__ E buf[2 * PNB * APPLY_CH];
  const int b = blockIdx.y, t = threadIdx.x, c0 = blockIdx.x * APPLY_CH;
  A += b * sA;
  const int* aff = piv + b * sP + aff_at;
  const int na = aff[0];
  for (int e = t; e < na * APPLY_CH; e += PT) {
    const int a = e / APPLY_CH, c = c0 + e % APPLY_CH;
    if (c < n) buf[e] = A[(long long)aff[1 + 2 * PNB + a] * lda + c];
  }
  __syncthreads();
  for (int e = t; e < na * APPLY_CH; e += PT) {
    const int a = e / APPLY_CH, c = c0 + e % APPLY_CH;
    if (c < n) A[(long long)aff[1 + a] * lda + c] = buf[e];
  }
}

// Solve L21 U11 = A21 for the rows below the (factored, moved) pivot block,
// one thread per row.
constexpr int FIN_T = 128;
template <typename E>
__global__ void __launch_bounds__(FIN_T) k_tp_finish(E* A, int lda, long long sA, int n, int j0) {
  __shared__ E U[PNB][PNB + 1];
  const int b = blockIdx.y, t = threadIdx.x;
  A += b * sA;
  for (int e = t; e < PNB * PNB; e += FIN_T) U[e / PNB][e % PNB] = A[(long long)(j0 + e / PNB) * lda + j0 + e % PNB];
  __syncthreads();
  const int r = j0 + PNB + blockIdx.x * FIN_T + t;
  if (r >= n) return;
  E* row = A + (long long)r * lda + j0;
  E x[PNB];
#pragma unroll
  for (int c = 0; c < PNB; ++c) x[c] = row[c];
#pragma unroll
  for (int c = 0; c < PNB; ++c) {
#pragma unroll
    for (int i = 0; i < c; ++i) x[c] = fmsc(x[c], x[i], U[i][c]);
    if (el<E>::mag2(U[c][c]) > 0.0) x[c] = el<E>::div(x[c], U[c][c]);
  }
#pragma unroll
  for (int c = 0; c < PNB; ++c) row[c] = x[c];
}

void set_smem_once(const void* f, size_t bytes) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> done;  // (kernel, device)
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  for (auto& d : done)
    if (d.first == f && d.second == dev) return;
  cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  done.emplace_back(f, dev);
}

size_t small_smem_elems(int m, int nb) {
  return (size_t)std::max(m * (nb + 1), std::min(m, 2 * nb) * APPLY_CH);
}

}  // namespace

template <typename E>
void lu_panel(cudaStream_t s, E* A, int lda, long long sA, int n, int j0, int nb, int* piv, long long sP, int* info,
              int batch) {
  const int m = n - j0;
  const size_t tile_bytes = (size_t)PR * (PNB + 1) * sizeof(E);
  if (m <= PR) {
    set_smem_once((const void*)k_panel_small<E>, tile_bytes);
    const size_t bytes = small_smem_elems(m, nb) * sizeof(E);
    k_panel_small<E><<<batch, PT, bytes, s>>>(A, lda, sA, n, j0, nb, piv, sP, info);
    HS_COUNT_LAUNCH();
    return;
  }
  // tournament (nb == PNB here: only the last panel is narrower, and it is short)
  set_smem_once((const void*)k_tp_select<E>, tile_bytes);
  int sets = (m + PR - 1) / PR, total = 0;
  for (int k = sets; k > 1; k = (k * nb + PR - 1) / PR) total += k * nb;  // lists of the non-final rounds
  const int aff_off = total;
  int in_off = -1, nin = 0, out_off = 0;
  for (;;) {
    const int fin = sets == 1;
    k_tp_select<E><<<dim3(sets, batch), PT, tile_bytes, s>>>(A, lda, sA, n, j0, nb, piv, sP, info, in_off, nin,
                                                             out_off, fin, aff_off);
    HS_COUNT_LAUNCH();
    if (fin) break;
    in_off = out_off;
    nin = sets * nb;
    out_off += nin;
    sets = (nin + PR - 1) / PR;
  }
  k_tp_apply<E><<<dim3((n + APPLY_CH - 1) / APPLY_CH, batch), PT, 0, s>>>(A, lda, sA, n, piv, sP,
                                                                          j0 + nb + aff_off);
  HS_COUNT_LAUNCH();
  k_tp_finish<E><<<dim3((m - PNB + FIN_T - 1) / FIN_T, batch), FIN_T, 0, s>>>(A, lda, sA, n, j0);
  HS_COUNT_LAUNCH();
}

template void lu_panel<double>(cudaStream_t, double*, int, long long, int, int, int, int*, long long, int*, int);
template void lu_panel<double2>(cudaStream_t, double2*, int, long long, int, int, int, int*, long long, int*, int);
template void lu_panel<float>(cudaStream_t, float*, int, long long, int, int, int, int*, long long, int*, int);
template void lu_panel<float2>(cudaStream_t, float2*, int, long long, int, int, int, int*, long long, int*, int);

}  // namespace hs
