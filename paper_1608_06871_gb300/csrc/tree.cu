// Merges of impedance-to-impedance maps up the quadtree and the sweeps down
// it (Sec. 2: "recursive merging" of "impedance-to-impedance" maps; O(N^{3/2})
// factorisation, then O(N log N) per right-hand side).
//
// For children alpha, beta with ItI maps R^a, R^b, exterior nodes "1" (alpha)
// and "2" (beta) and the shared interface "3" (same nodes, opposite normals):
// continuity of u and of the flux makes the incoming impedance on each side of
// the interface the negative of the outgoing one on the other.  Eliminating
// the interface gives
//   f3a = X f,   X = W [B33 A31, -B32],  W = (I - B33 A33)^{-1}
//   f3b = Z f,   Z = -[A31, 0] - A33 X
//   R   = blockdiag(A11, B22) + [A13 X ; B23 Z]
// where A = R^a, B = R^b restricted to the index sets.  The level routines
// build these with batched gathers, GEMMs and LU factorisations over all
// parent boxes of the level.
#include "tree.cuh"

namespace hs {

namespace {
__device__ __forceinline__ int src_child(int v) { return v >> 20; }
__device__ __forceinline__ int src_local(int v) { return v & 0xFFFFF; }

// A33 = R^a[I3a, I3a], B33 = R^b[I3b, I3b], M = I.
__global__ void k_gather_33(const double2* __restrict__ Rc, int nc, const int* __restrict__ alpha,
                            const int* __restrict__ beta, const int* __restrict__ I3a, const int* __restrict__ I3b,
                            int ni, double2* __restrict__ A33, double2* __restrict__ B33, double2* __restrict__ M) {
  const int b = blockIdx.y;
  const long long nn = (long long)ni * ni;
  const double2* Ra = Rc + (long long)alpha[b] * nc * nc;
  const double2* Rb = Rc + (long long)beta[b] * nc * nc;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / ni), c = (int)(e % ni);
    A33[b * nn + e] = Ra[(long long)I3a[r] * nc + I3a[c]];
    B33[b * nn + e] = Rb[(long long)I3b[r] * nc + I3b[c]];
    M[b * nn + e] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
}

// XZ top = Bb = [0, B32] (columns of beta-sourced parent nodes), XZ bottom = Aa = [A31, 0].
__global__ void k_gather_XZ(const double2* __restrict__ Rc, int nc, const int* __restrict__ alpha,
                            const int* __restrict__ beta, const int* __restrict__ I3a, const int* __restrict__ I3b,
                            const int* __restrict__ src, int ni, int np, double2* __restrict__ XZ) {
  const int b = blockIdx.y;
  const long long tot = 2LL * ni * np;
  const double2* Ra = Rc + (long long)alpha[b] * nc * nc;
  const double2* Rb = Rc + (long long)beta[b] * nc * nc;
  double2* out = XZ + b * tot;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / np), c = (int)(e % np);
    int sv = src[c];
    double2 v = make_double2(0.0, 0.0);
    if (r < ni) {
      if (src_child(sv) == 1) v = Rb[(long long)I3b[r] * nc + src_local(sv)];
    } else {
      if (src_child(sv) == 0) v = Ra[(long long)I3a[r - ni] * nc + src_local(sv)];
    }
    out[e] = v;
  }
}

// U2 rows: alpha-sourced parent node -> [A13 row, 0], beta-sourced -> [0, B23 row].
__global__ void k_gather_U2(const double2* __restrict__ Rc, int nc, const int* __restrict__ alpha,
                            const int* __restrict__ beta, const int* __restrict__ I3a, const int* __restrict__ I3b,
                            const int* __restrict__ src, int ni, int np, double2* __restrict__ U2) {
  const int b = blockIdx.y;
  const long long tot = (long long)np * 2 * ni;
  const double2* Ra = Rc + (long long)alpha[b] * nc * nc;
  const double2* Rb = Rc + (long long)beta[b] * nc * nc;
  double2* out = U2 + b * tot;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / (2 * ni)), c = (int)(e % (2 * ni));
    int sv = src[r];
    double2 v = make_double2(0.0, 0.0);
    if (c < ni) {
      if (src_child(sv) == 0) v = Ra[(long long)src_local(sv) * nc + I3a[c]];
    } else {
      if (src_child(sv) == 1) v = Rb[(long long)src_local(sv) * nc + I3b[c - ni]];
    }
    out[e] = v;
  }
}

// Rp = blockdiag(A11, B22) in the parent's node order.
__global__ void k_gather_diag(const double2* __restrict__ Rc, int nc, const int* __restrict__ alpha,
                              const int* __restrict__ beta, const int* __restrict__ src, int np,
                              double2* __restrict__ Rp) {
  const int b = blockIdx.y;
  const long long tot = (long long)np * np;
  const double2* Ra = Rc + (long long)alpha[b] * nc * nc;
  const double2* Rb = Rc + (long long)beta[b] * nc * nc;
  double2* out = Rp + b * tot;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / np), c = (int)(e % np);
    int sr = src[r], sc = src[c];
    double2 v = make_double2(0.0, 0.0);
    if (src_child(sr) == src_child(sc)) {
      const double2* Rx = src_child(sr) == 0 ? Ra : Rb;
      v = Rx[(long long)src_local(sr) * nc + src_local(sc)];
    }
    out[e] = v;
  }
}

// Children's incoming impedances from the parent's (exterior nodes) and the
// interface values T3 = [f3a; f3b].
__global__ void k_scatter_down(const double2* __restrict__ Fp, const double2* __restrict__ T3,
                               const int* __restrict__ alpha, const int* __restrict__ beta,
                               const int* __restrict__ src, const int* __restrict__ I3a,
                               const int* __restrict__ I3b, int nc, int ni, int np, int nrhs,
                               double2* __restrict__ Fc) {
  const int b = blockIdx.y;
  const long long rows = np + 2LL * ni;
  const long long tot = rows * nrhs;
  const int ca = alpha[b], cb = beta[b];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / nrhs), j = (int)(e % nrhs);
    if (r < np) {
      int sv = src[r];
      int child = src_child(sv) == 0 ? ca : cb;
      Fc[((long long)child * nc + src_local(sv)) * nrhs + j] = Fp[((long long)b * np + r) * nrhs + j];
    } else {
      int t = r - np;
      double2 v = T3[((long long)b * 2 * ni + t) * nrhs + j];
      if (t < ni)
        Fc[((long long)ca * nc + I3a[t]) * nrhs + j] = v;
      else
        Fc[((long long)cb * nc + I3b[t - ni]) * nrhs + j] = v;
    }
  }
}

// Adjoint: children's adjoint impedance loads.  MU[b] holds [Wt; la3] with
// Wt = M^{-T} lambda_ta and la3 = B33^T Wt - lambda_tb; alpha's interface gets
// la3, beta's gets -Wt, exterior nodes copy the parent's.
__global__ void k_scatter_adj(const double2* __restrict__ Lp, const double2* __restrict__ MU,
                              const int* __restrict__ alpha, const int* __restrict__ beta,
                              const int* __restrict__ src, const int* __restrict__ I3a,
                              const int* __restrict__ I3b, int nc, int ni, int np, int nrhs,
                              double2* __restrict__ Lc) {
  const int b = blockIdx.y;
  const long long rows = np + 2LL * ni;
  const long long tot = rows * nrhs;
  const int ca = alpha[b], cb = beta[b];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / nrhs), j = (int)(e % nrhs);
    if (r < np) {
      int sv = src[r];
      int child = src_child(sv) == 0 ? ca : cb;
      Lc[((long long)child * nc + src_local(sv)) * nrhs + j] = Lp[((long long)b * np + r) * nrhs + j];
    } else {
      int t = r - np;
      if (t < ni) {
        Lc[((long long)cb * nc + I3b[t]) * nrhs + j] = -MU[((long long)b * 2 * ni + t) * nrhs + j];
      } else {
        Lc[((long long)ca * nc + I3a[t - ni]) * nrhs + j] = MU[((long long)b * 2 * ni + t) * nrhs + j];
      }
    }
  }
}

inline unsigned grid_for(long long n, int per_block, int cap = 4096) {
  long long g = (n + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}
}  // namespace

void merge_level(cudaStream_t s, const Level& L, const double2* Rc, int* info) {
  const int ni = L.ni, np = L.np, nc = L.nc, nb = L.nbox;
  const long long nn = (long long)ni * ni, xz = 2LL * ni * np, pp = (long long)np * np;
  const double2 one = make_double2(1.0, 0.0), mone = make_double2(-1.0, 0.0), zero = make_double2(0.0, 0.0);
  k_gather_33<<<dim3(grid_for(nn, 256), nb), 256, 0, s>>>(Rc, nc, L.d_alpha, L.d_beta, L.d_I3a, L.d_I3b, ni, L.A33,
                                                          L.B33, L.M);
  HS_COUNT_LAUNCH();
  k_gather_XZ<<<dim3(grid_for(xz, 256), nb), 256, 0, s>>>(Rc, nc, L.d_alpha, L.d_beta, L.d_I3a, L.d_I3b, L.d_src, ni,
                                                          np, L.XZ);
  HS_COUNT_LAUNCH();
  k_gather_U2<<<dim3(grid_for(xz, 256), nb), 256, 0, s>>>(Rc, nc, L.d_alpha, L.d_beta, L.d_I3a, L.d_I3b, L.d_src, ni,
                                                          np, L.U2);
  HS_COUNT_LAUNCH();
  k_gather_diag<<<dim3(grid_for(pp, 256), nb), 256, 0, s>>>(Rc, nc, L.d_alpha, L.d_beta, L.d_src, np, L.R);
  HS_COUNT_LAUNCH();
  // M = I - B33 A33
  gemm<double2, double2, double2>(s, OP_N, OP_N, ni, ni, ni, mone, L.B33, ni, nn, L.A33, ni, nn, one, L.M, ni, nn, nb);
  // top = B33 * bottom - top  (V = B33 Aa - Bb)
  gemm<double2, double2, double2>(s, OP_N, OP_N, ni, np, ni, one, L.B33, ni, nn, L.XZ + nn * 0 + (long long)ni * np,
                                  np, xz, mone, L.XZ, np, xz, nb);
  lu_factor<double2>(s, L.M, ni, nn, ni, L.Mpiv, ni, info, nb);
  // X = M^{-1} V (top half)
  lu_solve<double2>(s, OP_N, L.M, ni, nn, ni, L.Mpiv, ni, L.XZ, np, xz, np, nb);
  // bottom = -A33 X - bottom  (Z = -Aa - A33 X)
  gemm<double2, double2, double2>(s, OP_N, OP_N, ni, np, ni, mone, L.A33, ni, nn, L.XZ, np, xz, mone,
                                  L.XZ + (long long)ni * np, np, xz, nb);
  // R = blockdiag + U2 [X; Z]
  gemm<double2, double2, double2>(s, OP_N, OP_N, np, np, 2 * ni, one, L.U2, 2 * ni, (long long)np * 2 * ni, L.XZ, np,
                                  xz, one, L.R, np, pp, nb);
  (void)zero;
}

void sweep_down_level(cudaStream_t s, const Level& L, const double2* Fp, double2* T3, double2* Fc, int nrhs) {
  const int ni = L.ni, np = L.np, nb = L.nbox;
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  gemm<double2, double2, double2>(s, OP_N, OP_N, 2 * ni, nrhs, np, one, L.XZ, np, 2LL * ni * np, Fp, nrhs,
                                  (long long)np * nrhs, zero, T3, nrhs, 2LL * ni * nrhs, nb);
  long long tot = ((long long)np + 2LL * ni) * nrhs;
  k_scatter_down<<<dim3(grid_for(tot, 256), nb), 256, 0, s>>>(Fp, T3, L.d_alpha, L.d_beta, L.d_src, L.d_I3a, L.d_I3b,
                                                              L.nc, ni, np, nrhs, Fc);
  HS_COUNT_LAUNCH();
}

void sweep_adjoint_level(cudaStream_t s, const Level& L, const double2* Lp, double2* MU, double2* Lc, int nrhs) {
  const int ni = L.ni, np = L.np, nb = L.nbox;
  const long long nn = (long long)ni * ni, mu = 2LL * ni * nrhs;
  const double2 one = make_double2(1.0, 0.0), mone = make_double2(-1.0, 0.0), zero = make_double2(0.0, 0.0);
  // [mu_a; mu_b] = U2^T lambda_p ;  lambda_tb = mu_b
  gemm<double2, double2, double2>(s, OP_T, OP_N, 2 * ni, nrhs, np, one, L.U2, 2 * ni, (long long)np * 2 * ni, Lp,
                                  nrhs, (long long)np * nrhs, zero, MU, nrhs, mu, nb);
  // lambda_ta = mu_a - A33^T lambda_tb
  gemm<double2, double2, double2>(s, OP_T, OP_N, ni, nrhs, ni, mone, L.A33, ni, nn, MU + (long long)ni * nrhs, nrhs,
                                  mu, one, MU, nrhs, mu, nb);
  // Wt = M^{-T} lambda_ta
  lu_solve<double2>(s, OP_T, L.M, ni, nn, ni, L.Mpiv, ni, MU, nrhs, mu, nrhs, nb);
  // la3 = B33^T Wt - lambda_tb
  gemm<double2, double2, double2>(s, OP_T, OP_N, ni, nrhs, ni, one, L.B33, ni, nn, MU, nrhs, mu, mone,
                                  MU + (long long)ni * nrhs, nrhs, mu, nb);
  long long tot = ((long long)np + 2LL * ni) * nrhs;
  k_scatter_adj<<<dim3(grid_for(tot, 256), nb), 256, 0, s>>>(Lp, MU, L.d_alpha, L.d_beta, L.d_src, L.d_I3a, L.d_I3b,
                                                             L.nc, ni, np, nrhs, Lc);
  HS_COUNT_LAUNCH();
}

}  // namespace hs
