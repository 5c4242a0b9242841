// Merges of impedance-to-impedance maps up the quadtree and the sweeps down
// it (Sec. 2: "recursive merging" of "impedance-to-impedance" maps; O(N^{3/2})
// factorisation, then O(N log N) per right-hand side).
//
// For children alpha, beta with ItI maps R^a, R^b, exterior nodes "1" (alpha)
// and "2" (beta) and the shared interface "3" (same nodes, opposite normals):
// continuity of u and of the flux makes the incoming impedance on each side of
// the interface the negative of the outgoing one on the other (plus the
// interface residual terms s_a, s_b when the continuity rows have a right-hand
// side).  Eliminating the interface gives
//   f3a = X f + t_a,   X = W [B33 A31, -B32],  W = (I - B33 A33)^{-1}
//   f3b = Z f + t_b,   Z = -[A31, 0] - A33 X
//   R   = blockdiag(A11, B22) + [A13 X ; B23 Z]
//   t_a = W (B33 (h3a - s_b) - (h3b - s_a)),   t_b = -A33 t_a - (h3a - s_b)
//   h   = [h1a + A13 t_a ; h2b + B23 t_b]      (particular outgoing impedance)
// where A = R^a, B = R^b restricted to the index sets and h the children's
// particular outgoing impedances (body loads).  The level routines do this
// with batched gathers, GEMMs and LU factorisations over all parents of a level.
#include <type_traits>

#include "tree.cuh"

namespace hs {

namespace {
__device__ __forceinline__ int src_child(int v) { return v >> 20; }
__device__ __forceinline__ int src_local(int v) { return v & 0xFFFFF; }

template <typename C> __device__ __forceinline__ C czero() { return el<C>::zero(); }

// A33 = R^a[I3a, I3a], B33 = R^b[I3b, I3b], M = I.
template <typename C>
__global__ void k_gather_33(const C* __restrict__ Rc, int nc, const int* __restrict__ alpha,
                            const int* __restrict__ beta, const int* __restrict__ I3a, const int* __restrict__ I3b,
                            int ni, C* __restrict__ A33, C* __restrict__ B33, C* __restrict__ M) {
  const int b = blockIdx.y;
  const long long nn = (long long)ni * ni;
  const C* Ra = Rc + (long long)alpha[b] * nc * nc;
  const C* Rb = Rc + (long long)beta[b] * nc * nc;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / ni), c = (int)(e % ni);
    A33[b * nn + e] = Ra[(long long)I3a[r] * nc + I3a[c]];
    B33[b * nn + e] = Rb[(long long)I3b[r] * nc + I3b[c]];
    M[b * nn + e] = r == c ? el<C>::one() : czero<C>();
  }
}

// XZ top = Bb = [0, B32] (columns of beta-sourced parent nodes), XZ bottom = Aa = [A31, 0].
template <typename C>
__global__ void k_gather_XZ(const C* __restrict__ Rc, int nc, const int* __restrict__ alpha,
                            const int* __restrict__ beta, const int* __restrict__ I3a, const int* __restrict__ I3b,
                            const int* __restrict__ src, int ni, int np, C* __restrict__ XZ) {
  const int b = blockIdx.y;
  const long long tot = 2LL * ni * np;
  const C* Ra = Rc + (long long)alpha[b] * nc * nc;
  const C* Rb = Rc + (long long)beta[b] * nc * nc;
  C* out = XZ + b * tot;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / np), c = (int)(e % np);
    int sv = src[c];
    C v = czero<C>();
    if (r < ni) {
      if (src_child(sv) == 1) v = Rb[(long long)I3b[r] * nc + src_local(sv)];
    } else {
      if (src_child(sv) == 0) v = Ra[(long long)I3a[r - ni] * nc + src_local(sv)];
    }
    out[e] = v;
  }
}

// U2 rows: alpha-sourced parent node r (< n1) -> A13 row, beta-sourced -> B23 row.
template <typename C>
__global__ void k_gather_U2(const C* __restrict__ Rc, int nc, const int* __restrict__ alpha,
                            const int* __restrict__ beta, const int* __restrict__ I3a, const int* __restrict__ I3b,
                            const int* __restrict__ src, int ni, int np, C* __restrict__ U2) {
  const int b = blockIdx.y;
  const long long tot = (long long)np * ni;
  const C* Ra = Rc + (long long)alpha[b] * nc * nc;
  const C* Rb = Rc + (long long)beta[b] * nc * nc;
  C* out = U2 + b * tot;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / ni), c = (int)(e % ni);
    int sv = src[r];
    out[e] = src_child(sv) == 0 ? Ra[(long long)src_local(sv) * nc + I3a[c]] : Rb[(long long)src_local(sv) * nc + I3b[c]];
  }
}

// Rp = blockdiag(A11, B22) in the parent's node order.
template <typename C>
__global__ void k_gather_diag(const C* __restrict__ Rc, int nc, const int* __restrict__ alpha,
                              const int* __restrict__ beta, const int* __restrict__ src, int np, C* __restrict__ Rp) {
  const int b = blockIdx.y;
  const long long tot = (long long)np * np;
  const C* Ra = Rc + (long long)alpha[b] * nc * nc;
  const C* Rb = Rc + (long long)beta[b] * nc * nc;
  C* out = Rp + b * tot;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / np), c = (int)(e % np);
    int sr = src[r], sc = src[c];
    C v = czero<C>();
    if (src_child(sr) == src_child(sc)) {
      const C* Rx = src_child(sr) == 0 ? Ra : Rb;
      v = Rx[(long long)src_local(sr) * nc + src_local(sc)];
    }
    out[e] = v;
  }
}

// Children's incoming impedances from the parent's (exterior nodes) and the
// interface values T3 = [f3a; f3b].
template <typename C>
__global__ void k_scatter_down(const C* __restrict__ Fp, const C* __restrict__ T3, const int* __restrict__ alpha,
                               const int* __restrict__ beta, const int* __restrict__ src, const int* __restrict__ I3a,
                               const int* __restrict__ I3b, int nc, int ni, int np, int nrhs, C* __restrict__ Fc) {
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
      C v = T3[((long long)b * 2 * ni + t) * nrhs + j];
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
template <typename C>
__global__ void k_scatter_adj(const C* __restrict__ Lp, const C* __restrict__ MU, const int* __restrict__ alpha,
                              const int* __restrict__ beta, const int* __restrict__ src, const int* __restrict__ I3a,
                              const int* __restrict__ I3b, int nc, int ni, int np, int nrhs, C* __restrict__ Lc) {
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

// Transpose of k_scatter_down: the children's adjoint impedance loads Lc give
// the adjoint of the interface impedances MU = [Lc_alpha(I3a); Lc_beta(I3b)]
// and the exterior part of the parent's, Lp(r) = Lc(child of r).
template <typename C>
__global__ void k_gather_adj_up(const C* __restrict__ Lc, const int* __restrict__ alpha, const int* __restrict__ beta,
                                const int* __restrict__ src, const int* __restrict__ I3a, const int* __restrict__ I3b,
                                int nc, int ni, int np, int nrhs, C* __restrict__ MU, C* __restrict__ Lp) {
  const int b = blockIdx.y;
  const long long rows = np + 2LL * ni;
  const long long tot = rows * nrhs;
  const int ca = alpha[b], cb = beta[b];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / nrhs), j = (int)(e % nrhs);
    if (r < np) {
      int sv = src[r];
      int child = src_child(sv) == 0 ? ca : cb;
      Lp[((long long)b * np + r) * nrhs + j] = Lc[((long long)child * nc + src_local(sv)) * nrhs + j];
    } else {
      int t = r - np;
      C v = t < ni ? Lc[((long long)ca * nc + I3a[t]) * nrhs + j] : Lc[((long long)cb * nc + I3b[t - ni]) * nrhs + j];
      MU[((long long)b * 2 * ni + t) * nrhs + j] = v;
    }
  }
}

// Upward gather: TT top := h3b - s_a, TT bottom := h3a - s_b, Hp := children's
// exterior particular impedances in the parent's order.
template <typename C>
__global__ void k_gather_up(const C* __restrict__ Hc, const C* __restrict__ S3, const int* __restrict__ alpha,
                            const int* __restrict__ beta, const int* __restrict__ src, const int* __restrict__ I3a,
                            const int* __restrict__ I3b, int nc, int ni, int np, int nrhs, C* __restrict__ TT,
                            C* __restrict__ Hp) {
  const int b = blockIdx.y;
  const long long rows = np + 2LL * ni;
  const long long tot = rows * nrhs;
  const int ca = alpha[b], cb = beta[b];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / nrhs), j = (int)(e % nrhs);
    if (r < np) {
      int sv = src[r];
      int child = src_child(sv) == 0 ? ca : cb;
      Hp[((long long)b * np + r) * nrhs + j] = Hc[((long long)child * nc + src_local(sv)) * nrhs + j];
    } else {
      int t = r - np;
      C v;
      C sres = czero<C>();
      if (t < ni) {  // h3b - s_a
        v = Hc[((long long)cb * nc + I3b[t]) * nrhs + j];
        if (S3) sres = S3[((long long)b * 2 * ni + t) * nrhs + j];
      } else {       // h3a - s_b
        v = Hc[((long long)ca * nc + I3a[t - ni]) * nrhs + j];
        if (S3) sres = S3[((long long)b * 2 * ni + t) * nrhs + j];
      }
      TT[((long long)b * 2 * ni + t) * nrhs + j] = v - sres;
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

template <typename C> void merge_level(cudaStream_t s, const LevelMaps& L, const LevelOps<C>& O, const C* Rc, int* info) {
  const int ni = L.ni, np = L.np, nc = L.nc, nb = L.nbox;
  const long long nn = (long long)ni * ni, xz = 2LL * ni * np, pp = (long long)np * np;
  const C one = el<C>::one(), mone = -el<C>::one();
  k_gather_33<C><<<dim3(grid_for(nn, 256), nb), 256, 0, s>>>(Rc, nc, L.d_alpha, L.d_beta, L.d_I3a, L.d_I3b, ni, O.A33,
                                                             O.B33, O.M);
  HS_COUNT_LAUNCH();
  k_gather_XZ<C><<<dim3(grid_for(xz, 256), nb), 256, 0, s>>>(Rc, nc, L.d_alpha, L.d_beta, L.d_I3a, L.d_I3b, L.d_src,
                                                             ni, np, O.XZ);
  HS_COUNT_LAUNCH();
  k_gather_U2<C><<<dim3(grid_for((long long)np * ni, 256), nb), 256, 0, s>>>(Rc, nc, L.d_alpha, L.d_beta, L.d_I3a,
                                                                               L.d_I3b, L.d_src, ni, np, O.U2);
  HS_COUNT_LAUNCH();
  constexpr bool kInv = std::is_same<C, float2>::value;  // FP32 factors keep W explicitly
  if (!kInv) {
    k_gather_diag<C><<<dim3(grid_for(pp, 256), nb), 256, 0, s>>>(Rc, nc, L.d_alpha, L.d_beta, L.d_src, np, O.R);
    HS_COUNT_LAUNCH();
  }
  // M = I - B33 A33
  gemm<C, C, C>(s, OP_N, OP_N, ni, ni, ni, mone, O.B33, ni, nn, O.A33, ni, nn, one, O.M, ni, nn, nb);
  // top = B33 * bottom - top  (V = B33 Aa - Bb)
  gemm<C, C, C>(s, OP_N, OP_N, ni, np, ni, one, O.B33, ni, nn, O.XZ + (long long)ni * np, np, xz, mone, O.XZ, np, xz,
                nb);
  lu_factor<C>(s, O.M, ni, nn, ni, O.Mpiv, ni, info, nb);
  if constexpr (kInv) {
    // W = M^{-1} explicitly (the sweeps then apply it with one GEMM per
    // level); R is free until its diagonal blocks are gathered and stages W
    // and then X = W V
    const C zero = el<C>::zero();
    lu_inverse<C>(s, O.M, ni, nn, ni, O.Mpiv, ni, O.R, ni, pp, nb);
    cudaMemcpy2DAsync(O.M, nn * sizeof(C), O.R, pp * sizeof(C), nn * sizeof(C), nb, cudaMemcpyDeviceToDevice,
                      s);
    gemm<C, C, C>(s, OP_N, OP_N, ni, np, ni, one, O.M, ni, nn, O.XZ, np, xz, zero, O.R, np, pp, nb);
    cudaMemcpy2DAsync(O.XZ, xz * sizeof(C), O.R, pp * sizeof(C), (size_t)ni * np * sizeof(C), nb,
                      cudaMemcpyDeviceToDevice, s);
    k_gather_diag<C><<<dim3(grid_for(pp, 256), nb), 256, 0, s>>>(Rc, nc, L.d_alpha, L.d_beta, L.d_src, np, O.R);
    HS_COUNT_LAUNCH();
  } else {
    // X = M^{-1} V (top half)
    lu_solve<C>(s, OP_N, O.M, ni, nn, ni, O.Mpiv, ni, O.XZ, np, xz, np, nb);
  }
  // bottom = -A33 X - bottom  (Z = -Aa - A33 X)
  gemm<C, C, C>(s, OP_N, OP_N, ni, np, ni, mone, O.A33, ni, nn, O.XZ, np, xz, mone, O.XZ + (long long)ni * np, np, xz,
                nb);
  // R rows of alpha's exterior += A13 X ; rows of beta's exterior += B23 Z
  const int n1 = L.n1, n2 = np - L.n1;
  const long long su = (long long)np * ni;
  gemm<C, C, C>(s, OP_N, OP_N, n1, np, ni, one, O.U2, ni, su, O.XZ, np, xz, one, O.R, np, pp, nb);
  gemm<C, C, C>(s, OP_N, OP_N, n2, np, ni, one, O.U2 + (long long)n1 * ni, ni, su, O.XZ + (long long)ni * np, np, xz,
                one, O.R + (long long)n1 * np, np, pp, nb);
}

template <typename C>
void sweep_down_level(cudaStream_t s, const LevelMaps& L, const LevelOps<C>& O, const C* Fp, C* T3, C* Fc, int nrhs,
                      bool t3_loaded) {
  const int ni = L.ni, np = L.np, nb = L.nbox;
  const C one = el<C>::one(), zero = el<C>::zero();
  gemm<C, C, C>(s, OP_N, OP_N, 2 * ni, nrhs, np, one, O.XZ, np, 2LL * ni * np, Fp, nrhs, (long long)np * nrhs,
                t3_loaded ? one : zero, T3, nrhs, 2LL * ni * nrhs, nb);
  long long tot = ((long long)np + 2LL * ni) * nrhs;
  k_scatter_down<C><<<dim3(grid_for(tot, 256), nb), 256, 0, s>>>(Fp, T3, L.d_alpha, L.d_beta, L.d_src, L.d_I3a,
                                                                 L.d_I3b, L.nc, ni, np, nrhs, Fc);
  HS_COUNT_LAUNCH();
}

template <typename C>
void sweep_adjoint_level(cudaStream_t s, const LevelMaps& L, const LevelOps<C>& O, const C* Lp, C* MU, C* Lc,
                         int nrhs, bool w_explicit, bool mu_loaded) {
  const int ni = L.ni, np = L.np, nb = L.nbox;
  const long long nn = (long long)ni * ni, mu = 2LL * ni * nrhs;
  const C one = el<C>::one(), mone = -el<C>::one(), zero = el<C>::zero();
  // mu_a = A13^T lambda_1, mu_b = B23^T lambda_2 ;  lambda_tb = mu_b  (added to the
  // adjoint of the particular interface impedances when MU holds it on entry)
  const int n1 = L.n1, n2 = np - L.n1;
  const long long su = (long long)np * ni, sl = (long long)np * nrhs;
  const C b0 = mu_loaded ? one : zero;
  gemm<C, C, C>(s, OP_T, OP_N, ni, nrhs, n1, one, O.U2, ni, su, Lp, nrhs, sl, b0, MU, nrhs, mu, nb);
  gemm<C, C, C>(s, OP_T, OP_N, ni, nrhs, n2, one, O.U2 + (long long)n1 * ni, ni, su, Lp + (long long)n1 * nrhs, nrhs,
                sl, b0, MU + (long long)ni * nrhs, nrhs, mu, nb);
  // lambda_ta = mu_a - A33^T lambda_tb
  gemm<C, C, C>(s, OP_T, OP_N, ni, nrhs, ni, mone, O.A33, ni, nn, MU + (long long)ni * nrhs, nrhs, mu, one, MU, nrhs,
                mu, nb);
  // Wt = M^{-T} lambda_ta  (M = I - B33 A33 factored, or W = M^{-1} kept explicitly)
  if (w_explicit) {
    // Lc (written only by the final scatter) holds the product meanwhile
    const long long tw = (long long)ni * nrhs;
    gemm<C, C, C>(s, OP_T, OP_N, ni, nrhs, ni, one, O.M, ni, nn, MU, nrhs, mu, zero, Lc, nrhs, tw, nb);
    cudaMemcpy2DAsync(MU, (size_t)mu * sizeof(C), Lc, (size_t)tw * sizeof(C), (size_t)tw * sizeof(C), nb,
                      cudaMemcpyDeviceToDevice, s);
  } else {
    lu_solve<C>(s, OP_T, O.M, ni, nn, ni, O.Mpiv, ni, MU, nrhs, mu, nrhs, nb);
  }
  // la3 = B33^T Wt - lambda_tb
  gemm<C, C, C>(s, OP_T, OP_N, ni, nrhs, ni, one, O.B33, ni, nn, MU, nrhs, mu, mone, MU + (long long)ni * nrhs, nrhs,
                mu, nb);
  long long tot = ((long long)np + 2LL * ni) * nrhs;
  k_scatter_adj<C><<<dim3(grid_for(tot, 256), nb), 256, 0, s>>>(Lp, MU, L.d_alpha, L.d_beta, L.d_src, L.d_I3a,
                                                                L.d_I3b, L.nc, ni, np, nrhs, Lc);
  HS_COUNT_LAUNCH();
}

template <typename C>
void sweep_adjoint_up_level(cudaStream_t s, const LevelMaps& L, const LevelOps<C>& O, const C* Lc, C* MU, C* Lp,
                            int nrhs) {
  const int ni = L.ni, np = L.np, nb = L.nbox;
  long long tot = ((long long)np + 2LL * ni) * nrhs;
  k_gather_adj_up<C><<<dim3(grid_for(tot, 256), nb), 256, 0, s>>>(Lc, L.d_alpha, L.d_beta, L.d_src, L.d_I3a, L.d_I3b,
                                                                  L.nc, ni, np, nrhs, MU, Lp);
  HS_COUNT_LAUNCH();
  // Lp += [X; Z]^T MU  (the interface impedances were [X; Z] f + [t_a; t_b])
  gemm<C, C, C>(s, OP_T, OP_N, np, nrhs, 2 * ni, el<C>::one(), O.XZ, np, 2LL * ni * np, MU, nrhs, 2LL * ni * nrhs,
                el<C>::one(), Lp, nrhs, (long long)np * nrhs, nb);
}

template <typename C>
void sweep_up_level(cudaStream_t s, const LevelMaps& L, const LevelOps<C>& O, const C* Hc, C* S3, C* TT, C* Hp,
                    int nrhs) {
  const int ni = L.ni, np = L.np, nb = L.nbox;
  const long long nn = (long long)ni * ni, tt = 2LL * ni * nrhs;
  const C one = el<C>::one(), mone = -el<C>::one();
  long long tot = ((long long)np + 2LL * ni) * nrhs;
  k_gather_up<C><<<dim3(grid_for(tot, 256), nb), 256, 0, s>>>(Hc, S3, L.d_alpha, L.d_beta, L.d_src, L.d_I3a, L.d_I3b,
                                                              L.nc, ni, np, nrhs, TT, Hp);
  HS_COUNT_LAUNCH();
  // top := B33 (h3a - s_b) - (h3b - s_a);  t_a = W top
  gemm<C, C, C>(s, OP_N, OP_N, ni, nrhs, ni, one, O.B33, ni, nn, TT + (long long)ni * nrhs, nrhs, tt, mone, TT, nrhs,
                tt, nb);
  if constexpr (std::is_same<C, float2>::value) {
    // M holds W explicitly: t_a = W top through S3 (consumed by the gather)
    gemm<C, C, C>(s, OP_N, OP_N, ni, nrhs, ni, one, O.M, ni, nn, TT, nrhs, tt, el<C>::zero(), S3, nrhs, tt, nb);
    cudaMemcpy2DAsync(TT, tt * sizeof(C), S3, tt * sizeof(C), (size_t)ni * nrhs * sizeof(C), nb,
                      cudaMemcpyDeviceToDevice, s);
  } else {
    lu_solve<C>(s, OP_N, O.M, ni, nn, ni, O.Mpiv, ni, TT, nrhs, tt, nrhs, nb);
  }
  // bottom := -A33 t_a - (h3a - s_b) = t_b
  gemm<C, C, C>(s, OP_N, OP_N, ni, nrhs, ni, mone, O.A33, ni, nn, TT, nrhs, tt, mone, TT + (long long)ni * nrhs, nrhs,
                tt, nb);
  // Hp rows of alpha's exterior += A13 t_a ; rows of beta's exterior += B23 t_b
  const int n1 = L.n1, n2 = np - L.n1;
  const long long su = (long long)np * ni, sh = (long long)np * nrhs;
  gemm<C, C, C>(s, OP_N, OP_N, n1, nrhs, ni, one, O.U2, ni, su, TT, nrhs, tt, one, Hp, nrhs, sh, nb);
  gemm<C, C, C>(s, OP_N, OP_N, n2, nrhs, ni, one, O.U2 + (long long)n1 * ni, ni, su, TT + (long long)ni * nrhs, nrhs, tt,
                one, Hp + (long long)n1 * nrhs, nrhs, sh, nb);
}

template <typename C>
__global__ void k_permute_rows(const C* __restrict__ src, const int* __restrict__ idx, int nrows, int ncols,
                               C* __restrict__ dst) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nrows * ncols) return;
  int r = (int)(e / ncols), c = (int)(e % ncols);
  dst[e] = src[(long long)idx[r] * ncols + c];
}

template <typename C>
__global__ void k_permute_square(const C* __restrict__ src, const int* __restrict__ idx, int n, C* __restrict__ dst) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  int r = (int)(e / n), c = (int)(e % n);
  dst[e] = src[(long long)idx[r] * n + idx[c]];
}

template <typename C> void permute_rows(cudaStream_t s, const C* src, const int* idx, int nrows, int ncols, C* dst) {
  long long n = (long long)nrows * ncols;
  k_permute_rows<C><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, idx, nrows, ncols, dst);
  HS_COUNT_LAUNCH();
}

template <typename C> void permute_square(cudaStream_t s, const C* src, const int* idx, int n, C* dst) {
  long long m = (long long)n * n;
  k_permute_square<C><<<(unsigned)((m + 255) / 256), 256, 0, s>>>(src, idx, n, dst);
  HS_COUNT_LAUNCH();
}

#define HS_INST(C)                                                                                                     \
  template void merge_level<C>(cudaStream_t, const LevelMaps&, const LevelOps<C>&, const C*, int*);                  \
  template void sweep_down_level<C>(cudaStream_t, const LevelMaps&, const LevelOps<C>&, const C*, C*, C*, int, bool); \
  template void sweep_adjoint_level<C>(cudaStream_t, const LevelMaps&, const LevelOps<C>&, const C*, C*, C*, int, bool, \
                                       bool);                                                                        \
  template void sweep_adjoint_up_level<C>(cudaStream_t, const LevelMaps&, const LevelOps<C>&, const C*, C*, C*, int);  \
  template void sweep_up_level<C>(cudaStream_t, const LevelMaps&, const LevelOps<C>&, const C*, C*, C*, C*, int);       \
  template void permute_rows<C>(cudaStream_t, const C*, const int*, int, int, C*);                                  \
  template void permute_square<C>(cudaStream_t, const C*, const int*, int, C*);
HS_INST(double2)
HS_INST(float2)
#undef HS_INST

}  // namespace hs
