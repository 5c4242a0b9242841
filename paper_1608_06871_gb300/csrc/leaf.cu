// Leaf-level kernels: the band-limited contrast on the leaf grids (Sec. 3.2,
// eq. sineseries, Definition of E_k) and the per-leaf spectral collocation
// operators of the direct solver (Sec. 2: K x K Chebyshev grids, K = 16).
//
// Leaf-local orderings (shared with tree.cu and hs_api.cu through tree.cuh):
//   interior node (a, b), 1 <= a, b <= 14:      r = (a-1)*14 + (b-1)       (196)
//   edge nodes in boundary order S, E, N, W,
//   each side by increasing coordinate:         e = side*14 + (t-1)        (56)
//   S: (a, 0)   E: (15, b)   N: (a, 15)   W: (0, b)
// The 4 corner nodes are not unknowns of the discretisation.
#include "tree.cuh"

namespace hs {

__constant__ double c_D1[16 * 16];  // Chebyshev-Lobatto differentiation on [-1, 1]

void upload_cheb_diff(const double* D1, cudaStream_t s) {
  cudaMemcpyToSymbolAsync(c_D1, D1, sizeof(double) * 256, 0, cudaMemcpyHostToDevice, s);
}

// s[m-1][g] = sin(m pi (x_g + 1) / 2) for the leaf-grid coordinates x_g (length ng).
__global__ void k_sine_table(const double* __restrict__ xg, int ng, int S, double* __restrict__ out) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int m = blockIdx.y + 1;
  if (g >= ng) return;
  out[(long long)(m - 1) * ng + g] = sinpi(0.5 * m * (xg[g] + 1.0));
}

// Scatter the global node grid Qg[gx][gy] (gx = ix*16 + a) into the leaf layout
// q[leaf][a][b] and flag 1 - q <= 0 or NaN.
__global__ void k_grid_to_leaves(const double* __restrict__ Qg, int nL, double* __restrict__ q, int* __restrict__ bad) {
  const int n16 = nL * 16;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n16 * n16) return;
  int gx = (int)(idx / n16), gy = (int)(idx % n16);
  int ix = gx / 16, a = gx % 16, iy = gy / 16, b = gy % 16;
  double v = Qg[idx];
  q[(((long long)(iy * nL + ix)) * 16 + a) * 16 + b] = v;
  if (!(1.0 - v > 0.0)) atomicExch(bad, 1);
}

__global__ void k_check_q(const double* __restrict__ q, long long n, int* __restrict__ bad) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(1.0 - q[i] > 0.0)) atomicExch(bad, 1);
}

__device__ __forceinline__ int edge_index(int a, int b) {
  if (b == 0) return a - 1;         // S
  if (a == 15) return 14 + b - 1;   // E
  if (b == 15) return 28 + a - 1;   // N
  return 42 + b - 1;                // W
}

// Assemble, per leaf, the blocks of the leaf system (interior PDE rows and the
// outward normal derivative at the edge nodes), computed in FP64 and stored in T:
//   Aii (196x196), Aie (196x56): rows of  Lap_h u + k^2 (1 - q) u  at interior nodes,
//   Ni (56x196), NiT = Ni^T (196x56), Ne (56x56): outward normal derivative rows.
template <typename T>
__global__ void __launch_bounds__(256) k_leaf_assemble(const double* __restrict__ q, int leaf0,
                                                       const double* __restrict__ kp, double h,
                                                       T* __restrict__ Aii, T* __restrict__ Aie, T* __restrict__ Ni,
                                                       T* __restrict__ NiT, T* __restrict__ Ne) {
  const int lb = blockIdx.x;  // leaf within the chunk
  const double k = *kp;       // read on the device, so that a captured build serves every k
  const double* ql = q + (long long)(leaf0 + lb) * 256;
  Aii += (long long)lb * NI * NI;
  Aie += (long long)lb * NI * NE;
  Ni += (long long)lb * NE * NI;
  NiT += (long long)lb * NI * NE;
  Ne += (long long)lb * NE * NE;
  __shared__ double Dx[16][16], D2[16][16];
  const double sc = 2.0 / h;
  for (int e = threadIdx.x; e < 256; e += blockDim.x) Dx[e / 16][e % 16] = c_D1[e] * sc;
  __syncthreads();
  for (int e = threadIdx.x; e < 256; e += blockDim.x) {
    int i = e / 16, j = e % 16;
    double s = 0.0;
    for (int c = 0; c < 16; ++c) s += Dx[i][c] * Dx[c][j];
    D2[i][j] = s;
  }
  for (int e = threadIdx.x; e < NI * NI; e += blockDim.x) Aii[e] = T(0);
  for (int e = threadIdx.x; e < NI * NE; e += blockDim.x) { Aie[e] = T(0); Ni[e] = T(0); NiT[e] = T(0); }
  for (int e = threadIdx.x; e < NE * NE; e += blockDim.x) Ne[e] = T(0);
  __syncthreads();
  // interior rows: one thread per row (every entry but the diagonal gets one term)
  for (int r = threadIdx.x; r < NI; r += blockDim.x) {
    const int a = r / 14 + 1, b = r % 14 + 1;
    T* row = Aii + (long long)r * NI;
    T* rowe = Aie + (long long)r * NE;
    for (int c = 1; c <= 14; ++c) {
      if (c != a) row[(c - 1) * 14 + (b - 1)] = T(D2[a][c]);  // d2/dx2 along the x-line through (a, b)
      if (c != b) row[(a - 1) * 14 + (c - 1)] = T(D2[b][c]);  // d2/dy2 along the y-line
    }
    double dg = D2[a][a];
    dg += D2[b][b];
    dg += k * k * (1.0 - ql[a * 16 + b]);
    row[r] = T(dg);
    rowe[edge_index(0, b)] = T(D2[a][0]);
    rowe[edge_index(15, b)] = T(D2[a][15]);
    rowe[edge_index(a, 0)] = T(D2[b][0]);
    rowe[edge_index(a, 15)] = T(D2[b][15]);
  }
  // normal-derivative rows: one thread per edge node (one term per entry)
  for (int e = threadIdx.x; e < NE; e += blockDim.x) {
    const int side = e / 14, t = e % 14 + 1;
    T* nrow = Ni + (long long)e * NI;
    T* erow = Ne + (long long)e * NE;
    for (int c = 0; c < 16; ++c) {
      int a, b;
      double w;
      switch (side) {
        case 0: a = t; b = c; w = -Dx[0][c]; break;    // S: -d/dy at (t, 0)
        case 1: a = c; b = t; w = Dx[15][c]; break;    // E: +d/dx at (15, t)
        case 2: a = t; b = c; w = Dx[15][c]; break;    // N: +d/dy at (t, 15)
        default: a = c; b = t; w = -Dx[0][c]; break;   // W: -d/dx at (0, t)
      }
      bool interior = (a >= 1 && a <= 14 && b >= 1 && b <= 14);
      if (interior) {
        int rr = (a - 1) * 14 + (b - 1);
        nrow[rr] = T(w);
        NiT[(long long)rr * NE + e] = T(w);
      } else {
        erow[edge_index(a, b)] = T(w);  // never a corner: one coordinate is t in 1..14
      }
    }
  }
}

// K = T + i eta I (complex), Kinv = I.
template <typename T>
__global__ void k_make_K(const T* __restrict__ Tm, const double* __restrict__ kp, typename prec<T>::C* __restrict__ K,
                         typename prec<T>::C* __restrict__ Kinv, int nleaf) {
  using C = typename prec<T>::C;
  const double eta = *kp;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nleaf * NE * NE) return;
  int e = (int)(idx % (NE * NE));
  int r = e / NE, c = e % NE;
  C kv, iv;
  kv.x = Tm[idx];
  kv.y = r == c ? T(eta) : T(0);
  iv.x = r == c ? T(1) : T(0);
  iv.y = T(0);
  K[idx] = kv;
  Kinv[idx] = iv;
}

// R = I - 2 i eta Kinv (leaf impedance-to-impedance map); Ye = Kinv (edge rows of Y).
template <typename T>
__global__ void k_leaf_R(const typename prec<T>::C* __restrict__ Kinv, const double* __restrict__ kp,
                         typename prec<T>::C* __restrict__ R,
                         typename prec<T>::C* __restrict__ Y, int nleaf) {
  using C = typename prec<T>::C;
  const double eta = *kp;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nleaf * NE * NE) return;
  int lb = (int)(idx / (NE * NE));
  int e = (int)(idx % (NE * NE));
  int r = e / NE, c = e % NE;
  C v = Kinv[idx];
  // -2 i eta (x + i y) = 2 eta y - 2 i eta x
  C rv;
  rv.x = T((r == c ? 1.0 : 0.0) + 2.0 * eta * (double)v.y);
  rv.y = T(-2.0 * eta * (double)v.x);
  R[idx] = rv;
  Y[(long long)lb * NL * NE + (long long)(NI + r) * NE + c] = v;
}

template <typename T>
void leaf_build_chunk(cudaStream_t s, const double* q, int leaf0, int nleaf, double k, const double* d_k, double h,
                      LeafScratchT<T>& w, typename prec<T>::C* R, typename prec<T>::C* Y, typename prec<T>::C* Q,
                      int* info) {
  using C = typename prec<T>::C;
  const double eta = k;
  k_leaf_assemble<T><<<nleaf, 256, 0, s>>>(q, leaf0, d_k, h, w.Aii, w.Aie, w.Ni, w.NiT, w.Ne);
  HS_COUNT_LAUNCH();
  lu_factor<T>(s, w.Aii, NI, (long long)NI * NI, NI, w.piv, NI, info, nleaf);
  // X = Aii^{-1} Aie (Dirichlet-to-interior map), W = Aii^{-T} Ni^T (adjoint)
  if (w.Ainv && !Q) {
    // keep Aii^{-1} (the mixed path's particular solves use it); X by one GEMM
    // staged in NiT, whose transpose rows the path without adjoint never needs
    lu_inverse<T>(s, w.Aii, NI, (long long)NI * NI, NI, w.piv, NI, w.Ainv + (long long)leaf0 * NI * NI, NI,
                  (long long)NI * NI, nleaf);
    gemm<T, T, T>(s, OP_N, OP_N, NI, NE, NI, T(1), w.Ainv + (long long)leaf0 * NI * NI, NI, (long long)NI * NI, w.Aie,
                  NE, (long long)NI * NE, T(0), w.NiT, NE, (long long)NI * NE, nleaf);
    cudaMemcpyAsync(w.Aie, w.NiT, sizeof(T) * (size_t)nleaf * NI * NE, cudaMemcpyDeviceToDevice, s);
  } else {
    lu_solve<T>(s, OP_N, w.Aii, NI, (long long)NI * NI, NI, w.piv, NI, w.Aie, NE, (long long)NI * NE, NE, nleaf);
  }
  if (Q)  // W is needed only by the adjoint operator
    lu_solve<T>(s, OP_T, w.Aii, NI, (long long)NI * NI, NI, w.piv, NI, w.NiT, NE, (long long)NI * NE, NE, nleaf);
  // T = Ne - Ni X  (leaf Dirichlet-to-Neumann map), stored in Ne
  gemm<T, T, T>(s, OP_N, OP_N, NE, NE, NI, T(-1), w.Ni, NI, (long long)NE * NI, w.Aie, NE, (long long)NI * NE, T(1),
                w.Ne, NE, (long long)NE * NE, nleaf);
  {
    long long n = (long long)nleaf * NE * NE;
    k_make_K<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w.Ne, d_k, w.K, w.Kinv, nleaf);
    HS_COUNT_LAUNCH();
  }
  lu_factor<C>(s, w.K, NE, (long long)NE * NE, NE, w.pivK, NE, info, nleaf);
  lu_solve<C>(s, OP_N, w.K, NE, (long long)NE * NE, NE, w.pivK, NE, w.Kinv, NE, (long long)NE * NE, NE, nleaf);
  {
    long long n = (long long)nleaf * NE * NE;
    k_leaf_R<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w.Kinv, d_k, R, Y, nleaf);
    HS_COUNT_LAUNCH();
  }
  C m1 = el<C>::zero(), z0 = el<C>::zero(), ieta2 = el<C>::zero();
  m1.x = T(-1);
  ieta2.y = T(2.0 * eta);
  // interior rows of the solution operator: Yi = -X Kinv
  gemm<T, C, C>(s, OP_N, OP_N, NI, NE, NE, m1, w.Aie, NE, (long long)NI * NE, w.Kinv, NE, (long long)NE * NE, z0, Y,
                NE, (long long)NL * NE, nleaf);
  // adjoint body-load operator: Q = 2 i eta W Kinv^T (skipped when Q is NULL)
  if (Q)
    gemm<T, C, C>(s, OP_N, OP_T, NI, NE, NE, ieta2, w.NiT, NE, (long long)NI * NE, w.Kinv, NE, (long long)NE * NE, z0,
                  Q, NE, (long long)NI * NE, nleaf);
}

// Impedance form of the leaf (hs_config.leaf_impedance; FP64 and, with the
// particular-solution operator, mixed contexts): with the
// incoming impedance f = d_n u + i eta u prescribed on the edge nodes,
//   L [u_i; u_e] = [b; f],   L = [A_ii, A_ie; N_i, N_e + i eta I]   (252 x 252),
// the interior impedance problem, uniquely solvable at every k, where the
// Dirichlet block A_ii is singular at the leaf's Dirichlet eigenvalues
// (k sqrt(1 - q) h = pi sqrt(a^2 + b^2)).  Its Schur complement on the edge is
// K = N_e - N_i A_ii^{-1} A_ie + i eta I, so the outputs are the ones of the
// Dirichlet route: the solution operator Y = L^{-1} [0; I] (Y_e = K^{-1},
// Y_i = -X K^{-1}), R = I - 2 i eta Y_e, and the adjoint body-load operator
// Q = -2 i eta (L^{-T} [0; I])_i (= 2 i eta A_ii^{-T} N_i^T K^{-T}).  The mixed
// path keeps P = L^{-1} [I; 0] instead: a body load b gives the leaf solution
// P b (its refinement's particular solves) and the transposed solve P^T g (the
// adjoint's), where the Dirichlet route applies A_ii^{-1}, X and K^{-1}.
template <typename T>
__global__ void k_leaf_L(const T* __restrict__ Aii, const T* __restrict__ Aie, const T* __restrict__ Ni,
                         const T* __restrict__ Ne, const double* __restrict__ kp, typename prec<T>::C* __restrict__ L,
                         typename prec<T>::C* __restrict__ Y, typename prec<T>::C* __restrict__ Et,
                         typename prec<T>::C* __restrict__ Pp, int nleaf) {
  using C = typename prec<T>::C;
  const double eta = *kp;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nleaf * NL * NL) return;
  const int lb = (int)(idx / (NL * NL)), e = (int)(idx % (NL * NL));
  const int r = e / NL, c = e % NL;
  T v;
  if (r < NI) {
    v = c < NI ? Aii[((long long)lb * NI + r) * NI + c] : Aie[((long long)lb * NI + r) * NE + (c - NI)];
  } else {
    v = c < NI ? Ni[((long long)lb * NE + (r - NI)) * NI + c] : Ne[((long long)lb * NE + (r - NI)) * NE + (c - NI)];
  }
  C lv;
  lv.x = v;
  lv.y = (r >= NI && r == c) ? T(eta) : T(0);
  L[idx] = lv;
  C one, zero;
  one.x = T(1); one.y = T(0);
  zero.x = T(0); zero.y = T(0);
  if (c < NE) {  // right-hand sides [0; I] for Y and for L^T
    const C ev = (r >= NI && r - NI == c) ? one : zero;
    const long long o = ((long long)lb * NL + r) * NE + c;
    Y[o] = ev;
    if (Et) Et[o] = ev;
  }
  if (Pp && c < NI) Pp[((long long)lb * NL + r) * NI + c] = r == c ? one : zero;  // [I; 0]
}

// R = I - 2 i eta Y_e, Q = -2 i eta Et_i (Q optional).
template <typename T>
__global__ void k_leaf_RQ(const typename prec<T>::C* __restrict__ Y, const typename prec<T>::C* __restrict__ Et,
                          const double* __restrict__ kp, typename prec<T>::C* __restrict__ R,
                          typename prec<T>::C* __restrict__ Q, int nleaf) {
  using C = typename prec<T>::C;
  const double eta = *kp;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nleaf * NL * NE) return;
  const int lb = (int)(idx / (NL * NE)), e = (int)(idx % (NL * NE));
  const int r = e / NE, c = e % NE;
  if (r >= NI) {
    const C y = Y[idx];  // -2 i eta (x + i y) = 2 eta y - 2 i eta x
    C rv;
    rv.x = T((r - NI == c ? 1.0 : 0.0) + 2.0 * eta * (double)y.y);
    rv.y = T(-2.0 * eta * (double)y.x);
    R[((long long)lb * NE + (r - NI)) * NE + c] = rv;
  } else if (Q) {
    const C t = Et[idx];
    C qv;
    qv.x = T(2.0 * eta * (double)t.y);
    qv.y = T(-2.0 * eta * (double)t.x);
    Q[((long long)lb * NI + r) * NE + c] = qv;
  }
}

template <typename T>
void leaf_build_chunk_impedance(cudaStream_t s, const double* q, int leaf0, int nleaf, double k, const double* d_k,
                                double h, LeafScratchT<T>& w, typename prec<T>::C* R, typename prec<T>::C* Y,
                                typename prec<T>::C* Q, int* info) {
  using C = typename prec<T>::C;
  (void)k;
  k_leaf_assemble<T><<<nleaf, 256, 0, s>>>(q, leaf0, d_k, h, w.Aii, w.Aie, w.Ni, w.NiT, w.Ne);
  HS_COUNT_LAUNCH();
  C* Pp = w.P ? w.P + (long long)leaf0 * NL * NI : nullptr;
  {
    const long long n = (long long)nleaf * NL * NL;
    k_leaf_L<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w.Aii, w.Aie, w.Ni, w.Ne, d_k, w.L, Y, Q ? w.Et : nullptr,
                                                            Pp, nleaf);
    HS_COUNT_LAUNCH();
  }
  lu_factor<C>(s, w.L, NL, (long long)NL * NL, NL, w.pivL, NL, info, nleaf);
  lu_solve<C>(s, OP_N, w.L, NL, (long long)NL * NL, NL, w.pivL, NL, Y, NE, (long long)NL * NE, NE, nleaf);
  if (Q) lu_solve<C>(s, OP_T, w.L, NL, (long long)NL * NL, NL, w.pivL, NL, w.Et, NE, (long long)NL * NE, NE, nleaf);
  if (Pp) lu_solve<C>(s, OP_N, w.L, NL, (long long)NL * NL, NL, w.pivL, NL, Pp, NI, (long long)NL * NI, NI, nleaf);
  {
    const long long n = (long long)nleaf * NL * NE;
    k_leaf_RQ<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Y, w.Et, d_k, R, Q, nleaf);
    HS_COUNT_LAUNCH();
  }
}

template void leaf_build_chunk_impedance<double>(cudaStream_t, const double*, int, int, double, const double*, double,
                                                 LeafScratchT<double>&, double2*, double2*, double2*, int*);
template void leaf_build_chunk_impedance<float>(cudaStream_t, const double*, int, int, double, const double*, double,
                                                LeafScratchT<float>&, float2*, float2*, float2*, int*);

template void leaf_build_chunk<double>(cudaStream_t, const double*, int, int, double, const double*, double,
                                       LeafScratchT<double>&, double2*, double2*, double2*, int*);
template void leaf_build_chunk<float>(cudaStream_t, const double*, int, int, double, const double*, double,
                                      LeafScratchT<float>&, float2*, float2*, float2*, int*);

void sine_eval_grid(cudaStream_t s, const double* c, int S1, int S2, const double* xg, int nL, double* sx, double* sy,
                    double* T, double* Qg, double* q, int* bad) {
  const int n16 = nL * 16;
  dim3 g1((n16 + 127) / 128, S1), g2((n16 + 127) / 128, S2);
  k_sine_table<<<g1, 128, 0, s>>>(xg, n16, S1, sx);
  HS_COUNT_LAUNCH();
  k_sine_table<<<g2, 128, 0, s>>>(xg, n16, S2, sy);
  HS_COUNT_LAUNCH();
  // T[m1][gy] = sum_m2 c[m1][m2] sy[m2][gy];   Qg[gx][gy] = sum_m1 sx[m1][gx] T[m1][gy]
  gemm<double, double, double>(s, OP_N, OP_N, S1, n16, S2, 1.0, c, S2, 0, sy, n16, 0, 0.0, T, n16, 0, 1);
  gemm<double, double, double>(s, OP_T, OP_N, n16, n16, S1, 1.0, sx, n16, 0, T, n16, 0, 0.0, Qg, n16, 0, 1);
  long long n = (long long)n16 * n16;
  k_grid_to_leaves<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Qg, nL, q, bad);
  HS_COUNT_LAUNCH();
}

void check_q(cudaStream_t s, const double* q, long long n, int* bad) {
  k_check_q<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(q, n, bad);
  HS_COUNT_LAUNCH();
}

}  // namespace hs
