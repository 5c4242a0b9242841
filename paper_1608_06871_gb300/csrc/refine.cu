// Mixed-precision pieces: FP64 residuals of the discrete system and the FP32
// particular (body-load) solve at the leaves.
//
// The discrete system solved by the direct solver (Sec. 2) has three kinds of
// rows: the collocated PDE at interior leaf nodes, continuity of u and of the
// normal derivative at shared leaf edge nodes, and the exterior identity
// (D - I/2)(u - u_inc) = S (d_n u - d_n u_inc) at boundary nodes (Sec. 2,
// Remark).  With FP32 factors, the solution is refined in FP64: the residual
// of every row is computed here in FP64 from the current FP64 iterate (leaf
// layout [leaf][252][nrhs]) and fed to an FP32 solve for the correction.
#include "tree.cuh"

namespace hs {

namespace {

// Leaf-local unknown index of node (a, b) (never a corner).
__device__ __forceinline__ int lidx(int a, int b) {
  if (a >= 1 && a <= 14 && b >= 1 && b <= 14) return (a - 1) * 14 + (b - 1);
  if (b == 0) return NI + a - 1;
  if (a == 15) return NI + 14 + b - 1;
  if (b == 15) return NI + 28 + a - 1;
  return NI + 42 + b - 1;
}

__global__ void k_d2f(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

__global__ void k_f2d_add(const float2* __restrict__ a, double2* __restrict__ b, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_double2(b[i].x + (double)a[i].x, b[i].y + (double)a[i].y);
}

constexpr int RCH = 8;              // right-hand sides per block in the PDE residual
constexpr int RP_THREADS = 49 * RCH;  // one thread per (a, b) in 1..7 x 1..7 and right-hand side

// RP[leaf][r][j] = -(Lap_h u + k^2 (1 - q) u) at interior node r, for the FP64 iterate X.
// The second-derivative matrix D2 = (2/h)^2 D1 D1 of the Chebyshev points is
// centro-symmetric (D2[15-a][15-c] = D2[a][c]), so along a grid line with
// s_c = u_c + u_(15-c), d_c = u_c - u_(15-c) (c < 8) and E[a][c], O[a][c] the
// half sums and differences of D2[a][c] and D2[a][15-c]:
//   (D2 u)_a = sum_c E[a][c] s_c + O[a][c] d_c,  (D2 u)_(15-a) = the same with -O,
// half the FP64 multiply-adds of the plain row products (the FP64 pipe bounds
// this kernel).  Each thread forms the four mirror nodes (a, b), (15-a, b),
// (a, 15-b), (15-a, 15-b) of one right-hand side from the s, d of the two
// columns and two rows through them.
__global__ void __launch_bounds__(RP_THREADS) k_res_pde(const double2* __restrict__ X, const double* __restrict__ q,
                                                        const double* __restrict__ D1, double k, double h, int nrhs,
                                                        float2* __restrict__ RP) {
  __shared__ double Dx[16][16], D2r[8][16], E[8][8], O[8][8];
  extern __shared__ double2 rp_dyn[];  // u[NL][RCH], then sx, dx, sy, dy [14][8][RCH]
  auto u = reinterpret_cast<double2(*)[RCH]>(rp_dyn);
  auto sx = reinterpret_cast<double2(*)[8][RCH]>(rp_dyn + NL * RCH);
  auto dx = sx + 14, sy = sx + 28, dy = sx + 42;
  const int leaf = blockIdx.x, j0 = blockIdx.y * RCH, t = threadIdx.x;
  const int nj = min(RCH, nrhs - j0);
  const double sc = 2.0 / h;
  for (int e = t; e < 256; e += RP_THREADS) Dx[e / 16][e % 16] = D1[e] * sc;
  for (int e = t; e < NL * RCH; e += RP_THREADS) {
    const int r = e / RCH, j = e % RCH;
    u[r][j] = j < nj ? X[((long long)leaf * NL + r) * nrhs + j0 + j] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  // rows 1..7 of D2; the line sums and differences (x lines: column b = l + 1;
  // y lines: row a = l + 1)
  for (int e = t; e < 7 * 16; e += RP_THREADS) {
    const int a = e / 16 + 1, c = e % 16;
    double acc = 0.0;
    for (int m = 0; m < 16; ++m) acc = fma(Dx[a][m], Dx[m][c], acc);
    D2r[a][c] = acc;
  }
  for (int e = t; e < 2 * 14 * 8 * RCH; e += RP_THREADS) {
    const int j = e % RCH, c = (e / RCH) % 8, l = (e / (8 * RCH)) % 14, dir = e / (14 * 8 * RCH);
    if (dir == 0) {
      const double2 p = u[lidx(c, l + 1)][j], m = u[lidx(15 - c, l + 1)][j];
      sx[l][c][j] = p + m;
      dx[l][c][j] = p - m;
    } else {
      const double2 p = u[lidx(l + 1, c)][j], m = u[lidx(l + 1, 15 - c)][j];
      sy[l][c][j] = p + m;
      dy[l][c][j] = p - m;
    }
  }
  __syncthreads();
  for (int e = t; e < 7 * 8; e += RP_THREADS) {
    const int a = e / 8 + 1, c = e % 8;
    E[a][c] = 0.5 * (D2r[a][c] + D2r[a][15 - c]);
    O[a][c] = 0.5 * (D2r[a][c] - D2r[a][15 - c]);
  }
  __syncthreads();
  const int j = t % RCH, pr = t / RCH;
  if (j >= nj) return;
  const int a = pr / 7 + 1, b = pr % 7 + 1;  // a, b in 1..7; mirrors 15 - a, 15 - b
  double2 xe1 = make_double2(0.0, 0.0), xo1 = xe1, xe2 = xe1, xo2 = xe1;  // columns b, 15 - b
  double2 ye1 = xe1, yo1 = xe1, ye2 = xe1, yo2 = xe1;                     // rows a, 15 - a
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const double ea = E[a][c], oa = O[a][c], eb = E[b][c], ob = O[b][c];
    xe1 = xe1 + ea * sx[b - 1][c][j];
    xo1 = xo1 + oa * dx[b - 1][c][j];
    xe2 = xe2 + ea * sx[14 - b][c][j];
    xo2 = xo2 + oa * dx[14 - b][c][j];
    ye1 = ye1 + eb * sy[a - 1][c][j];
    yo1 = yo1 + ob * dy[a - 1][c][j];
    ye2 = ye2 + eb * sy[14 - a][c][j];
    yo2 = yo2 + ob * dy[14 - a][c][j];
  }
  const double* ql = q + (long long)leaf * 256;
  const double kk = k * k;
  // (A, B, x part, y part)
  const int An[4] = {a, 15 - a, a, 15 - a}, Bn[4] = {b, b, 15 - b, 15 - b};
  const double2 xp[4] = {xe1 + xo1, xe1 - xo1, xe2 + xo2, xe2 - xo2};
  const double2 yp[4] = {ye1 + yo1, ye2 + yo2, ye1 - yo1, ye2 - yo2};
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    const int A = An[n], B = Bn[n], r = (A - 1) * 14 + (B - 1);
    const double2 acc = xp[n] + yp[n] + (kk * (1.0 - ql[A * 16 + B])) * u[r][j];
    RP[((long long)leaf * NL + r) * nrhs + j0 + j] = make_float2((float)(-acc.x), (float)(-acc.y));
  }
}

// Outward normal derivative of leaf field U (leaf layout, FP64) at its edge
// node (a, b), right-hand side j.
__device__ double2 normal_deriv(const double2* __restrict__ U, int nrhs, int j, const double* __restrict__ D1,
                                double sc, int a, int b) {
  double2 acc = make_double2(0.0, 0.0);
  if (b == 0) {
    for (int c = 0; c < 16; ++c) acc = acc - (D1[c] * sc) * U[(long long)lidx(a, c) * nrhs + j];
  } else if (a == 15) {
    for (int c = 0; c < 16; ++c) acc = acc + (D1[15 * 16 + c] * sc) * U[(long long)lidx(c, b) * nrhs + j];
  } else if (b == 15) {
    for (int c = 0; c < 16; ++c) acc = acc + (D1[15 * 16 + c] * sc) * U[(long long)lidx(a, c) * nrhs + j];
  } else {
    for (int c = 0; c < 16; ++c) acc = acc - (D1[c] * sc) * U[(long long)lidx(c, b) * nrhs + j];
  }
  return acc;
}

// Interface residual terms of one merge level: for interface node t of parent
// b, with r_C = -(u_a - u_b) and r_F = -(d_n u_a + d_n u_b),
// S3[b][t] = r_F + i eta r_C (s_a) and S3[b][ni + t] = r_F - i eta r_C (s_b).
__global__ void k_res_iface(const double2* __restrict__ X, const double* __restrict__ D1, int nL, double h,
                            const double* __restrict__ kp, int horiz, int sx, int sy, int ni, int nbx_p, int nrhs,
                            float2* __restrict__ S3) {
  const int b = blockIdx.y;
  const double eta = *kp;
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)ni * nrhs) return;
  const int t = (int)(e / nrhs), j = (int)(e % nrhs);
  const int px = b % nbx_p, py = b / nbx_p;
  int la, lb, aa, ba, ab, bb;  // leaves and edge nodes on the alpha / beta side
  if (horiz) {
    const int x0 = px * 2 * sx, y0 = py * sy;
    const int ly = y0 + t / 14, node = t % 14 + 1;
    la = ly * nL + (x0 + sx - 1);
    lb = ly * nL + (x0 + sx);
    aa = 15; ba = node;  // alpha: east edge
    ab = 0; bb = node;   // beta: west edge
  } else {
    const int x0 = px * sx, y0 = py * 2 * sy;
    const int lx = x0 + t / 14, node = t % 14 + 1;
    la = (y0 + sy - 1) * nL + lx;
    lb = (y0 + sy) * nL + lx;
    aa = node; ba = 15;  // alpha: north edge
    ab = node; bb = 0;   // beta: south edge
  }
  const double sc = 2.0 / h;
  const double2* Ua = X + (long long)la * NL * nrhs;
  const double2* Ub = X + (long long)lb * NL * nrhs;
  double2 ua = Ua[(long long)lidx(aa, ba) * nrhs + j], ub = Ub[(long long)lidx(ab, bb) * nrhs + j];
  double2 na = normal_deriv(Ua, nrhs, j, D1, sc, aa, ba), nb2 = normal_deriv(Ub, nrhs, j, D1, sc, ab, bb);
  double2 rc = ub - ua;                 // -(u_a - u_b)
  double2 rf = -(na + nb2);
  // i eta rc = (-eta rc.y, eta rc.x)
  double2 sa = make_double2(rf.x - eta * rc.y, rf.y + eta * rc.x);
  double2 sbv = make_double2(rf.x + eta * rc.y, rf.y - eta * rc.x);
  S3[((long long)b * 2 * ni + t) * nrhs + j] = make_float2((float)sa.x, (float)sa.y);
  S3[((long long)b * 2 * ni + ni + t) * nrhs + j] = make_float2((float)sbv.x, (float)sbv.y);
}

// u and d_n u at the boundary nodes (root order: S, E, N, W, each by
// increasing coordinate) from the leaf fields.
__global__ void k_boundary_gather(const double2* __restrict__ X, const double* __restrict__ D1, int nL, double h,
                                  int nrhs, double2* __restrict__ ub, double2* __restrict__ psib) {
  const int nb = 56 * nL;
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nb * nrhs) return;
  const int jn = (int)(e / nrhs), j = (int)(e % nrhs);
  const int side = jn / (14 * nL), i = (jn % (14 * nL)) / 14, t = jn % 14 + 1;
  int leaf, a, b;
  switch (side) {
    case 0: leaf = i; a = t; b = 0; break;                       // S: leaf (i, 0)
    case 1: leaf = i * nL + (nL - 1); a = 15; b = t; break;      // E: leaf (nL-1, i)
    case 2: leaf = (nL - 1) * nL + i; a = t; b = 15; break;      // N: leaf (i, nL-1)
    default: leaf = i * nL; a = 0; b = t; break;                 // W: leaf (0, i)
  }
  const double2* U = X + (long long)leaf * NL * nrhs;
  ub[e] = U[(long long)lidx(a, b) * nrhs + j];
  psib[e] = normal_deriv(U, nrhs, j, D1, 2.0 / h, a, b);
}

// H = -2 i eta u_e^p (particular outgoing impedance) from the edge rows of Upart.
__global__ void k_leaf_h(const float2* __restrict__ Upart, int nleaf, const double* __restrict__ kp, int nrhs,
                         float2* __restrict__ H) {
  const double eta = *kp;
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nleaf * NE * nrhs) return;
  const int j = (int)(e % nrhs);
  const long long t = e / nrhs;
  const int r = (int)(t % NE), leaf = (int)(t / NE);
  float2 v = Upart[((long long)leaf * NL + NI + r) * nrhs + j];
  const float te = (float)(2.0 * eta);
  H[e] = make_float2(te * v.y, -te * v.x);  // -2 i eta (x + i y)
}

__global__ void k_scattered(const double2* __restrict__ ub, const double2* __restrict__ psib,
                            const double2* __restrict__ ui, const double2* __restrict__ dni, long long n,
                            double2* __restrict__ PS) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  PS[e] = ub[e] - ui[e];
  PS[n + e] = psib[e] - dni[e];
}

// Scattered boundary data [u - u_inc; d_n u - d_n u_inc] (root order) of an
// FP32 leaf field, in FP32; without the incident terms when sub_inc == 0 (a
// correction field).  Feeds the FP32 far field of one refinement pass.
__global__ void k_scattered32(const float2* __restrict__ U32, const double* __restrict__ D1, int nL, double h,
                              int nrhs, const double2* __restrict__ ui, const double2* __restrict__ dni, int sub_inc,
                              float2* __restrict__ PS) {
  const int nb = 56 * nL;
  const long long n = (long long)nb * nrhs;
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int jn = (int)(e / nrhs), j = (int)(e % nrhs);
  const int side = jn / (14 * nL), i = (jn % (14 * nL)) / 14, t = jn % 14 + 1;
  int leaf, a, b;
  switch (side) {
    case 0: leaf = i; a = t; b = 0; break;
    case 1: leaf = i * nL + (nL - 1); a = 15; b = t; break;
    case 2: leaf = (nL - 1) * nL + i; a = t; b = 15; break;
    default: leaf = i * nL; a = 0; b = t; break;
  }
  const float2* U = U32 + (long long)leaf * NL * nrhs;
  const float sc = (float)(2.0 / h);
  const int cpos = (a == 15 || b == 15) ? 15 : 0;
  const float sg = cpos == 15 ? 1.f : -1.f;
  float2 d = make_float2(0.f, 0.f);
  for (int c = 0; c < 16; ++c) {
    const float w = sg * (float)D1[cpos * 16 + c] * sc;
    const float2 v = (b == 0 || b == 15) ? U[(long long)lidx(a, c) * nrhs + j] : U[(long long)lidx(c, b) * nrhs + j];
    d = make_float2(d.x + w * v.x, d.y + w * v.y);
  }
  float2 u = U[(long long)lidx(a, b) * nrhs + j];
  if (sub_inc) {
    u = make_float2(u.x - (float)ui[e].x, u.y - (float)ui[e].y);
    d = make_float2(d.x - (float)dni[e].x, d.y - (float)dni[e].y);
  }
  PS[e] = u;
  PS[n + e] = d;
}

// DS = [D - I/2, -S] (nb x 2 nb): the exterior rows act on [u; d_n u] with one
// product; FP64 and FP32 copies.
__global__ void k_stack_ext(const double2* __restrict__ Dm, const double2* __restrict__ S, int nb,
                            double2* __restrict__ DS, float2* __restrict__ DS32) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2LL * nb * nb) return;
  const long long r = e / (2 * nb);
  const int c = (int)(e % (2 * nb));
  const double2 v = c < nb ? Dm[r * nb + c] : -S[r * nb + c - nb];
  DS[e] = v;
  DS32[e] = make_float2((float)v.x, (float)v.y);
}

// out[0] += sum |a|^2 (FP32 data, FP64 sums)
// out += sum |a|^2: a grid of a few blocks per SM strides over a, each block
// reduces its threads' FP64 partial sums and adds them with one atomic (an
// atomic per warp serialised on the one address for fields of 3e7 values).
constexpr int kNormBlocks = 4 * 152;
__global__ void __launch_bounds__(256) k_norm2_32(const float2* __restrict__ a, long long n, double* __restrict__ out) {
  __shared__ double red[8];
  double v = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 x = a[i];
    v += (double)x.x * x.x + (double)x.y * x.y;
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(out, v);
  }
}

// ---- adjoint refinement: transposed residual r = L - A^T Y -------------------
//
// Y holds the adjoint in the row space of the discrete system: Ypde at every
// interior leaf node (the PDE rows), per merge level the adjoints of the
// interface terms s_a = r_F + i eta r_C and s_b = r_F - i eta r_C (so that the
// continuity rows u_a - u_b and the flux rows d_n u_a + d_n u_b carry
// Y_C = i eta (Ys_a - Ys_b) and Y_F = Ys_a + Ys_b), and the exterior rows
// [D - I/2, -S] [u; d_n u] at the boundary nodes (through V = [D - I/2, -S]^T Yext).
// L is the receiver functional u_far(p) = A2[p] . [u; d_n u] at the boundary.
// Per leaf edge node the edge coefficients (Eu of the node's own u, En of its
// outward normal derivative) collect the interface and exterior terms; the
// kernel then applies the transposed leaf rows.

constexpr int ACH = 8;  // right-hand sides per block in the adjoint residual

__global__ void __launch_bounds__(256) k_adj_res(const double2* __restrict__ Ypde, const int4* __restrict__ desc,
                                                 const double2* __restrict__ Yif, const double2* __restrict__ A2,
                                                 const double2* __restrict__ V, const double* __restrict__ q,
                                                 const double* __restrict__ D1, double k, double h, double eta, int nb,
                                                 int nrhs, int first, float2* __restrict__ G) {
  __shared__ double D2[16][16], Dx[16][16];
  __shared__ double2 y[NI][ACH];
  __shared__ double2 eu[NE][ACH], en[NE][ACH];
  const int leaf = blockIdx.x, j0 = blockIdx.y * ACH;
  const int nj = min(ACH, nrhs - j0);
  const double sc = 2.0 / h;
  for (int e = threadIdx.x; e < 256; e += blockDim.x) Dx[e / 16][e % 16] = D1[e] * sc;
  if (!first)
    for (int e = threadIdx.x; e < NI * ACH; e += blockDim.x) {
      const int r = e / ACH, j = e % ACH;
      y[r][j] = j < nj ? Ypde[((long long)leaf * NI + r) * nrhs + j0 + j] : make_double2(0.0, 0.0);
    }
  for (int e = threadIdx.x; e < NE * ACH; e += blockDim.x) {
    const int r = e / ACH, j = e % ACH;
    double2 u = make_double2(0.0, 0.0), n = make_double2(0.0, 0.0);
    if (j < nj) {
      const int4 d = desc[leaf * NE + r];
      const long long p = j0 + j;
      if (d.z == 2) {  // boundary node d.x: u_far row minus the exterior rows' transpose
        u = A2[p * 2 * nb + d.x];
        n = A2[p * 2 * nb + nb + d.x];
        if (V) {
          u = u - V[(long long)d.x * nrhs + p];
          n = n - V[(long long)(nb + d.x) * nrhs + p];
        }
      } else if (!first) {  // interface node: d.x = (offset of its s_a row) / nrhs, d.y = ni
        const double2 sa = Yif[(long long)d.x * nrhs + p], sb = Yif[((long long)d.x + d.y) * nrhs + p];
        const double2 dd = sa - sb;
        const double2 yc = make_double2(-eta * dd.y, eta * dd.x);  // i eta (Ys_a - Ys_b)
        u = d.z == 0 ? -yc : yc;                                  // row u_a - u_b
        n = -(sa + sb);                                           // row d_n u_a + d_n u_b
      }
    }
    eu[r][j] = u;
    en[r][j] = n;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 256; e += blockDim.x) {
    const int i = e / 16, jj = e % 16;
    double s2 = 0.0;
    for (int c = 0; c < 16; ++c) s2 += Dx[i][c] * Dx[c][jj];
    D2[i][jj] = s2;
  }
  __syncthreads();
  const double* ql = q + (long long)leaf * 256;
  for (int e = threadIdx.x; e < NL * ACH; e += blockDim.x) {
    const int r = e / ACH, j = e % ACH;
    if (j >= nj) continue;
    int i, jy;  // x and y indices of unknown r
    if (r < NI) {
      i = r / 14 + 1;
      jy = r % 14 + 1;
    } else {
      const int ed = r - NI, side = ed / 14, t = ed % 14 + 1;
      switch (side) {
        case 0: i = t; jy = 0; break;    // S
        case 1: i = 15; jy = t; break;   // E
        case 2: i = t; jy = 15; break;   // N
        default: i = 0; jy = t; break;   // W
      }
    }
    double2 acc = make_double2(0.0, 0.0);
    if (!first) {  // transposed PDE rows of this leaf
      if (jy >= 1 && jy <= 14)
        for (int a = 1; a <= 14; ++a) acc = acc + D2[a][i] * y[(a - 1) * 14 + jy - 1][j];
      if (i >= 1 && i <= 14)
        for (int b = 1; b <= 14; ++b) acc = acc + D2[b][jy] * y[(i - 1) * 14 + b - 1][j];
      if (r < NI) acc = acc + (k * k * (1.0 - ql[i * 16 + jy])) * y[r][j];
    }
    double2 v = -acc;
    if (r >= NI) v = v + eu[r - NI][j];
    if (i >= 1 && i <= 14) {  // normal derivatives at the S and N nodes of column i
      v = v + (-Dx[0][jy]) * en[i - 1][j];
      v = v + Dx[15][jy] * en[28 + i - 1][j];
    }
    if (jy >= 1 && jy <= 14) {  // at the W and E nodes of row jy
      v = v + (-Dx[0][i]) * en[42 + jy - 1][j];
      v = v + Dx[15][i] * en[14 + jy - 1][j];
    }
    G[((long long)leaf * NL + r) * nrhs + j0 + j] = make_float2((float)v.x, (float)v.y);
  }
}

// Edge rows of the transposed leaf step: G_e += -2 i eta Hadj (the adjoint of
// the leaf's particular outgoing impedance h = -2 i eta u_e).
__global__ void k_leaf_hadj(const float2* __restrict__ H, int nleaf, double eta, int nrhs, float2* __restrict__ G) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nleaf * NE * nrhs) return;
  const int j = (int)(e % nrhs);
  const long long t = e / nrhs;
  const int r = (int)(t % NE), leaf = (int)(t / NE);
  const float2 v = H[e];
  const float te = (float)(2.0 * eta);
  float2* g = G + ((long long)leaf * NL + NI + r) * nrhs + j;
  *g = make_float2(g->x + te * v.y, g->y - te * v.x);
}

// Yif += [MU top; -MU bottom] for one level ([nbox][2 ni][nrhs]): the adjoints of
// s_a and s_b are Wt and -la3 of the transposed sweep.
__global__ void k_iface_adj_add(const float2* __restrict__ MU, int ni, int nrhs, long long n, double2* __restrict__ Y) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int t = (int)((e / nrhs) % (2 * ni));
  const float2 m = MU[e];
  const double sg = t < ni ? 1.0 : -1.0;
  Y[e] = make_double2(Y[e].x + sg * m.x, Y[e].y + sg * m.y);
}

inline unsigned blocks(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

void adjoint_residual(cudaStream_t s, const double2* Ypde, const int4* desc, const double2* Yif, const double2* A2,
                      const double2* V, const double* q, const double* D1, int nleaf, int nb, double k, double h,
                      double eta, int nrhs, bool first, float2* G) {
  dim3 g(nleaf, (nrhs + ACH - 1) / ACH);
  k_adj_res<<<g, 256, 0, s>>>(Ypde, desc, Yif, A2, V, q, D1, k, h, eta, nb, nrhs, first ? 1 : 0, G);
  HS_COUNT_LAUNCH();
}

void leaf_hadj(cudaStream_t s, const float2* H, int nleaf, double eta, int nrhs, float2* G) {
  long long n = (long long)nleaf * NE * nrhs;
  k_leaf_hadj<<<blocks(n), 256, 0, s>>>(H, nleaf, eta, nrhs, G);
  HS_COUNT_LAUNCH();
}

void iface_adj_add(cudaStream_t s, const float2* MU, int nbox, int ni, int nrhs, double2* Y) {
  long long n = (long long)nbox * 2 * ni * nrhs;
  k_iface_adj_add<<<blocks(n), 256, 0, s>>>(MU, ni, nrhs, n, Y);
  HS_COUNT_LAUNCH();
}

void convert_d2f(cudaStream_t s, const double2* a, float2* b, long long n) {
  k_d2f<<<blocks(n), 256, 0, s>>>(a, b, n);
  HS_COUNT_LAUNCH();
}

void convert_f2d_add(cudaStream_t s, const float2* a, double2* b, long long n) {
  k_f2d_add<<<blocks(n), 256, 0, s>>>(a, b, n);
  HS_COUNT_LAUNCH();
}

void residual_pde(cudaStream_t s, const double2* X, const double* q, const double* D1, int nleaf, double k, double h,
                  int nrhs, float2* RP) {
  dim3 g(nleaf, (nrhs + RCH - 1) / RCH);
  constexpr int bytes = (NL + 4 * 14 * 8) * RCH * (int)sizeof(double2);
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    cudaFuncSetAttribute(k_res_pde, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  k_res_pde<<<g, RP_THREADS, bytes, s>>>(X, q, D1, k, h, nrhs, RP);
  HS_COUNT_LAUNCH();
}

void residual_iface(cudaStream_t s, const LevelMaps& L, const double2* X, const double* D1, int nL, double h,
                    const double* d_k, int nrhs, float2* S3) {
  dim3 g(blocks((long long)L.ni * nrhs), L.nbox);
  k_res_iface<<<g, 256, 0, s>>>(X, D1, nL, h, d_k, L.horiz, L.sx, L.sy, L.ni, L.nbx_p, nrhs, S3);
  HS_COUNT_LAUNCH();
}

void boundary_gather(cudaStream_t s, const double2* X, const double* D1, int nL, double h, int nrhs, double2* ub,
                     double2* psib) {
  long long n = 56LL * nL * nrhs;
  k_boundary_gather<<<blocks(n), 256, 0, s>>>(X, D1, nL, h, nrhs, ub, psib);
  HS_COUNT_LAUNCH();
}

// Particular leaf solution for body loads b held in Upart rows 0..195 (FP32):
// w = Aii^{-1} b, u_e = -Kinv Ni w, u_i = w - X u_e, and h = -2 i eta u_e.
// With w.Ainv the first step is one GEMM into wtmp (NI x nrhs per leaf) and a
// copy back; otherwise triangular solves with the LU factors.
void leaf_particular(cudaStream_t s, const LeafScratchT<float>& w, int nleaf, const double* d_k, int nrhs, float2* Upart,
                     float2* H, float2* tmp, float2* wtmp) {
  const long long sU = (long long)NL * nrhs;
  const float2 one = make_float2(1.f, 0.f), mone = make_float2(-1.f, 0.f), zero = make_float2(0.f, 0.f);
  if (w.P) {  // impedance-form leaves: [u_i; u_e] = P b in one product (b staged in wtmp)
    cudaMemcpy2DAsync(wtmp, (size_t)NI * nrhs * sizeof(float2), Upart, sU * sizeof(float2),
                      (size_t)NI * nrhs * sizeof(float2), nleaf, cudaMemcpyDeviceToDevice, s);
    gemm<float2, float2, float2>(s, OP_N, OP_N, NL, nrhs, NI, one, w.P, NI, (long long)NL * NI, wtmp, nrhs,
                                 (long long)NI * nrhs, zero, Upart, nrhs, sU, nleaf);
    const long long n = (long long)nleaf * NE * nrhs;
    k_leaf_h<<<blocks(n), 256, 0, s>>>(Upart, nleaf, d_k, nrhs, H);
    HS_COUNT_LAUNCH();
    return;
  }
  if (w.Ainv && wtmp) {
    gemm<float, float2, float2>(s, OP_N, OP_N, NI, nrhs, NI, one, w.Ainv, NI, (long long)NI * NI, Upart, nrhs, sU,
                                zero, wtmp, nrhs, (long long)NI * nrhs, nleaf);
    cudaMemcpy2DAsync(Upart, sU * sizeof(float2), wtmp, (size_t)NI * nrhs * sizeof(float2),
                      (size_t)NI * nrhs * sizeof(float2), nleaf, cudaMemcpyDeviceToDevice, s);
  } else {
    // complex right-hand sides are solved as 2 nrhs real columns
    lu_solve<float>(s, OP_N, w.Aii, NI, (long long)NI * NI, NI, w.piv, NI, reinterpret_cast<float*>(Upart), 2 * nrhs,
                    2 * sU, 2 * nrhs, nleaf);
  }
  gemm<float, float2, float2>(s, OP_N, OP_N, NE, nrhs, NI, one, w.Ni, NI, (long long)NE * NI, Upart, nrhs, sU, zero,
                              tmp, nrhs, (long long)NE * nrhs, nleaf);
  gemm<float2, float2, float2>(s, OP_N, OP_N, NE, nrhs, NE, mone, w.Kinv, NE, (long long)NE * NE, tmp, nrhs,
                               (long long)NE * nrhs, zero, Upart + (long long)NI * nrhs, nrhs, sU, nleaf);
  gemm<float, float2, float2>(s, OP_N, OP_N, NI, nrhs, NE, mone, w.Aie, NE, (long long)NI * NE,
                              Upart + (long long)NI * nrhs, nrhs, sU, one, Upart, nrhs, sU, nleaf);
  long long n = (long long)nleaf * NE * nrhs;
  k_leaf_h<<<blocks(n), 256, 0, s>>>(Upart, nleaf, d_k, nrhs, H);
  HS_COUNT_LAUNCH();
}

void scattered32(cudaStream_t s, const float2* U32, const double* D1, int nL, double h, int nrhs, const double2* ui,
                 const double2* dni, bool sub_inc, float2* PS) {
  long long n = 56LL * nL * nrhs;
  k_scattered32<<<blocks(n), 256, 0, s>>>(U32, D1, nL, h, nrhs, ui, dni, sub_inc ? 1 : 0, PS);
  HS_COUNT_LAUNCH();
}

void stack_exterior(cudaStream_t s, const double2* Dm, const double2* S, int nb, double2* DS, float2* DS32) {
  k_stack_ext<<<blocks(2LL * nb * nb), 256, 0, s>>>(Dm, S, nb, DS, DS32);
  HS_COUNT_LAUNCH();
}

void norm2_32(cudaStream_t s, const float2* a, long long n, double* out) {
  if (n <= 0) return;
  k_norm2_32<<<(unsigned)std::min<long long>(kNormBlocks, (n + 255) / 256), 256, 0, s>>>(a, n, out);
  HS_COUNT_LAUNCH();
}

void scattered_data(cudaStream_t s, const double2* ub, const double2* psib, const double2* ui, const double2* dni,
                    long long n, double2* PS) {
  k_scattered<<<blocks(n), 256, 0, s>>>(ub, psib, ui, dni, n, PS);
  HS_COUNT_LAUNCH();
}

}  // namespace hs
