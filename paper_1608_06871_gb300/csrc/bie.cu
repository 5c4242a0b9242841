// Exterior coupling on the boundary of Omega (Sec. 2, Remark): the single and
// double layer operators
//   S phi(x) = int G(x,y) phi(y) ds_y,   D phi(x) = int dG/dn_y(x,y) phi(y) ds_y,
//   G(x,y) = (i/4) H_0^(1)(k |x-y|),
// discretised by Nystrom on the leaf-edge panels, the incident traces of the
// plane waves u_inc = exp(i k x.d) (Sec. 1), and Green's representation of the
// scattered field at the receivers x_p = R (cos theta_p, sin theta_p)
// (Sec. 1, the measured data u_far).
//
// Panel rule: each boundary panel (one leaf edge, length h) carries the 14
// interior Chebyshev-Lobatto nodes of the edge with Fejer's second-rule
// weights.  A target and a source panel within one panel length of each other
// use product integration of the exact kernel against the panel's Lagrange
// basis: Gauss-Legendre on intervals graded dyadically toward the point of the
// panel nearest the target (56 levels, so the innermost interval is below
// 2^-56 h), which resolves the logarithmic singularity of H_0.
//
// Combined-field rows (hs_config.bm_eta > 0): Green's identity alone is
// singular where k^2 is a Dirichlet eigenvalue of the square; its
// Burton-Miller combination with the normal-derivative identity
// T u_s = (K' + I/2) d_n u_s, coupling alpha = i eta / k, is solvable at every
// k.  K' has the kernel dG/dn_x; T = dD/dn_x comes from Maue's identity
// T phi = d/dt_x S(dphi/dt) + k^2 (n_x . n_y) S phi, with t the
// counter-clockwise tangent: the tangential-derivative kernel dG/dt_x is
// integrated like S and D on the near panels, and on the target's own panel as
// a principal value (its Cauchy part -sgn / (2 pi (s_x - s)) in closed form,
// the logarithmic remainder by the graded rule).
#include "tree.cuh"

namespace hs {

namespace {
constexpr int NGL = 16;    // Gauss-Legendre points per graded interval
constexpr int NLEV = 56;   // dyadic levels
constexpr int NPT = 14;    // panel nodes
constexpr int NEAR = 5;    // near panels per panel (itself and two on each side)
}  // namespace

__constant__ double c_glx[NGL], c_glw[NGL];
__constant__ double c_tnode[NPT], c_lagden[NPT];
__constant__ double c_dref[NPT * NPT];  // L_j'(t_l) on the panel nodes, [l][j]

void upload_quad_constants(const double* gl_x, const double* gl_w, const double* tnodes, const double* lagden,
                           const double* dref, cudaStream_t s) {
  cudaMemcpyToSymbolAsync(c_glx, gl_x, sizeof(double) * NGL, 0, cudaMemcpyHostToDevice, s);
  cudaMemcpyToSymbolAsync(c_glw, gl_w, sizeof(double) * NGL, 0, cudaMemcpyHostToDevice, s);
  cudaMemcpyToSymbolAsync(c_tnode, tnodes, sizeof(double) * NPT, 0, cudaMemcpyHostToDevice, s);
  cudaMemcpyToSymbolAsync(c_lagden, lagden, sizeof(double) * NPT, 0, cudaMemcpyHostToDevice, s);
  cudaMemcpyToSymbolAsync(c_dref, dref, sizeof(double) * NPT * NPT, 0, cudaMemcpyHostToDevice, s);
}

// +1 where a panel's tangent runs counter-clockwise (the outward normal turned
// by +90 degrees), -1 otherwise.
__device__ __forceinline__ double ccw_sign(double tx, double ty, double nx, double ny) {
  return (-ny * tx + nx * ty) > 0.0 ? 1.0 : -1.0;
}

// -(i k / 4) H_1(k r) / r: the common factor of dG/dn_x and dG/dt_x (times the
// projection of x - y on the target's normal or tangent).
__device__ __forceinline__ double2 h1_over_r(double k, double r) {
  const double z = k * r, c = 0.25 * k / r;
  return make_double2(c * y1(z), -c * j1(z));
}

// (i/4) H0(z) and (i k / 4) H1(z) * (an / r), H_n = J_n + i Y_n.
__device__ __forceinline__ double2 g_kernel(double z) { return make_double2(-0.25 * y0(z), 0.25 * j0(z)); }
__device__ __forceinline__ double2 dg_kernel(double z, double k, double an_over_r) {
  double s = 0.25 * k * an_over_r;
  return make_double2(-s * y1(z), s * j1(z));
}

__global__ void k_bie_plain(const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ nx,
                            const double* __restrict__ ny, const double* __restrict__ w, int nb, double k,
                            double2* __restrict__ S, double2* __restrict__ Dl) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nb * nb) return;
  int i = (int)(e / nb), j = (int)(e % nb);
  if (i == j) {
    S[e] = make_double2(0.0, 0.0);
    Dl[e] = make_double2(0.0, 0.0);
    return;
  }
  double dx = x[i] - x[j], dy = y[i] - y[j];
  double r = sqrt(dx * dx + dy * dy);
  double an = dx * nx[j] + dy * ny[j];
  double2 g = g_kernel(k * r), d = dg_kernel(k * r, k, an / r);
  S[e] = make_double2(g.x * w[j], g.y * w[j]);
  Dl[e] = make_double2(d.x * w[j], d.y * w[j]);
}

// One block per (target node, near-panel slot): product-integration weights of
// S and D against the 14 Lagrange basis polynomials of the source panel.
__global__ void __launch_bounds__(128) k_bie_near(const double* __restrict__ x, const double* __restrict__ y,
                                                  const int* __restrict__ panel, const double* __restrict__ p0x,
                                                  const double* __restrict__ p0y, const double* __restrict__ tx,
                                                  const double* __restrict__ ty, const double* __restrict__ pnx,
                                                  const double* __restrict__ pny, const int* __restrict__ nearp,
                                                  double h, double k, int nb, double2* __restrict__ S,
                                                  double2* __restrict__ Dl) {
  const int i = blockIdx.x;
  const int q = nearp[panel[i] * NEAR + blockIdx.y];
  if (q < 0) return;
  const double ax = x[i] - p0x[q], ay = y[i] - p0y[q];
  const double at = ax * tx[q] + ay * ty[q];
  const double an = ax * pnx[q] + ay * pny[q];  // exactly 0 for a target on the source's side
  const double sstar = fmin(fmax(at, 0.0), h);
  const double ov = at - sstar;
  double accS[2 * NPT], accD[2 * NPT];
#pragma unroll
  for (int j = 0; j < 2 * NPT; ++j) { accS[j] = 0.0; accD[j] = 0.0; }
  const int per_side = (NLEV + 1) * NGL;
  for (int p = threadIdx.x; p < 2 * per_side; p += blockDim.x) {
    const int side = p / per_side, rem = p % per_side;
    const int lev = rem / NGL, g = rem % NGL;
    const double d = side == 0 ? -sstar : h - sstar;
    if (d == 0.0) continue;
    const double hi = d * ldexp(1.0, -lev);
    const double lo = lev < NLEV ? 0.5 * hi : 0.0;
    const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
    const double sig = mid + half * c_glx[g];
    const double wq = fabs(half) * c_glw[g];
    const double dt = ov - sig;
    const double r = sqrt(an * an + dt * dt);
    double2 gk = g_kernel(k * r), dk = dg_kernel(k * r, k, an / r);
    // Lagrange basis at t = 2 s / h - 1 by prefix/suffix products
    const double tt = 2.0 * (sstar + sig) / h - 1.0;
    double pre[NPT], suf[NPT];
    pre[0] = 1.0;
    for (int j = 1; j < NPT; ++j) pre[j] = pre[j - 1] * (tt - c_tnode[j - 1]);
    suf[NPT - 1] = 1.0;
    for (int j = NPT - 2; j >= 0; --j) suf[j] = suf[j + 1] * (tt - c_tnode[j + 1]);
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
      double L = pre[j] * suf[j] / c_lagden[j] * wq;
      accS[2 * j] += gk.x * L;
      accS[2 * j + 1] += gk.y * L;
      accD[2 * j] += dk.x * L;
      accD[2 * j + 1] += dk.y * L;
    }
  }
  __shared__ double red[4][4 * NPT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 2 * NPT; ++j) {
    double a = accS[j], b = accD[j];
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      red[warp][j] = a;
      red[warp][2 * NPT + j] = b;
    }
  }
  __syncthreads();
  if (threadIdx.x < NPT) {
    int j = threadIdx.x;
    double sr = 0, si = 0, dr = 0, di = 0;
    for (int wv = 0; wv < 4; ++wv) {
      sr += red[wv][2 * j];
      si += red[wv][2 * j + 1];
      dr += red[wv][2 * NPT + 2 * j];
      di += red[wv][2 * NPT + 2 * j + 1];
    }
    long long o = (long long)i * nb + q * NPT + j;
    S[o] = make_double2(sr, si);
    Dl[o] = make_double2(dr, di);
  }
}

void bie_matrices(cudaStream_t s, const Boundary& B, double k, double2* S, double2* Dl) {
  long long n = (long long)B.nb * B.nb;
  k_bie_plain<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(B.x, B.y, B.nx, B.ny, B.w, B.nb, k, S, Dl);
  HS_COUNT_LAUNCH();
  k_bie_near<<<dim3(B.nb, NEAR), 128, 0, s>>>(B.x, B.y, B.panel, B.p0x, B.p0y, B.tx, B.ty, B.pnx, B.pny, B.near,
                                              B.h, k, B.nb, S, Dl);
  HS_COUNT_LAUNCH();
}

// Far entries of K' (kernel dG/dn_x) and H (kernel dG/dt_x, t_x the
// counter-clockwise tangent at the target) with the node weights; the near
// panels are overwritten by k_bie_near_nt.
__global__ void k_bie_plain_nt(const double* __restrict__ x, const double* __restrict__ y,
                               const double* __restrict__ nx, const double* __restrict__ ny,
                               const double* __restrict__ w, const int* __restrict__ panel,
                               const double* __restrict__ tx, const double* __restrict__ ty,
                               const double* __restrict__ pnx, const double* __restrict__ pny, int nb, double k,
                               double2* __restrict__ Kp, double2* __restrict__ H) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nb * nb) return;
  const int i = (int)(e / nb), j = (int)(e % nb);
  if (i == j) {
    Kp[e] = make_double2(0.0, 0.0);
    H[e] = make_double2(0.0, 0.0);
    return;
  }
  const int p = panel[i];
  const double sg = ccw_sign(tx[p], ty[p], pnx[p], pny[p]);
  const double dx = x[i] - x[j], dy = y[i] - y[j];
  const double r = sqrt(dx * dx + dy * dy);
  const double2 c = h1_over_r(k, r) * w[j];
  Kp[e] = c * (dx * nx[i] + dy * ny[i]);
  H[e] = c * (sg * (dx * tx[p] + dy * ty[p]));
}

// One block per (target node, near-panel slot), as k_bie_near: product
// integration of dG/dn_x and dG/dt_x against the source panel's Lagrange
// basis.  With x - y = dt tau_q + an n_q in the source panel's frame, the
// projections on the target's normal and tangent are dt (tau_q . n_x) +
// an (n_q . n_x) and the same with t_x.  On the target's own panel (an = 0,
// tau_q . n_x = 0, tau_q . t_x = sgn) K' vanishes and H is a principal value.
__global__ void __launch_bounds__(128) k_bie_near_nt(const double* __restrict__ x, const double* __restrict__ y,
                                                     const double* __restrict__ nx, const double* __restrict__ ny,
                                                     const int* __restrict__ panel, const double* __restrict__ p0x,
                                                     const double* __restrict__ p0y, const double* __restrict__ tx,
                                                     const double* __restrict__ ty, const double* __restrict__ pnx,
                                                     const double* __restrict__ pny, const int* __restrict__ nearp,
                                                     double h, double k, int nb, double2* __restrict__ Kp,
                                                     double2* __restrict__ H) {
  const int i = blockIdx.x, pi = panel[i];
  const int q = nearp[pi * NEAR + blockIdx.y];
  if (q < 0) return;
  const bool self = q == pi;
  const double sg = ccw_sign(tx[pi], ty[pi], pnx[pi], pny[pi]);
  const double txx = sg * tx[pi], txy = sg * ty[pi], nxi = nx[i], nyi = ny[i];
  const double cn1 = tx[q] * nxi + ty[q] * nyi, cn2 = pnx[q] * nxi + pny[q] * nyi;
  const double ct1 = tx[q] * txx + ty[q] * txy, ct2 = pnx[q] * txx + pny[q] * txy;
  const double ax = x[i] - p0x[q], ay = y[i] - p0y[q];
  const double at = ax * tx[q] + ay * ty[q];
  const double an = ax * pnx[q] + ay * pny[q];
  const double sstar = fmin(fmax(at, 0.0), h);
  const double ov = at - sstar;
  constexpr double inv2pi = 0.15915494309189533577;
  double accK[2 * NPT], accH[2 * NPT];
#pragma unroll
  for (int j = 0; j < 2 * NPT; ++j) { accK[j] = 0.0; accH[j] = 0.0; }
  const int per_side = (NLEV + 1) * NGL;
  for (int p = threadIdx.x; p < 2 * per_side; p += blockDim.x) {
    const int side = p / per_side, rem = p % per_side;
    const int lev = rem / NGL, g = rem % NGL;
    const double d = side == 0 ? -sstar : h - sstar;
    if (d == 0.0) continue;
    const double hi = d * ldexp(1.0, -lev);
    const double lo = lev < NLEV ? 0.5 * hi : 0.0;
    const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
    const double sig = mid + half * c_glx[g];
    const double wq = fabs(half) * c_glw[g];
    const double dt = ov - sig;
    const double r = sqrt(an * an + dt * dt);
    const double2 c = h1_over_r(k, r);
    const double2 kv = c * (dt * cn1 + an * cn2);
    double2 hv = c * (dt * ct1 + an * ct2);
    if (self) hv.x += sg * inv2pi / dt;  // minus the Cauchy part sg * (-1 / (2 pi dt))
    const double tt = 2.0 * (sstar + sig) / h - 1.0;
    double pre[NPT], suf[NPT];
    pre[0] = 1.0;
    for (int j = 1; j < NPT; ++j) pre[j] = pre[j - 1] * (tt - c_tnode[j - 1]);
    suf[NPT - 1] = 1.0;
    for (int j = NPT - 2; j >= 0; --j) suf[j] = suf[j + 1] * (tt - c_tnode[j + 1]);
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
      const double L = pre[j] * suf[j] / c_lagden[j] * wq;
      accK[2 * j] += kv.x * L;
      accK[2 * j + 1] += kv.y * L;
      accH[2 * j] += hv.x * L;
      accH[2 * j + 1] += hv.y * L;
    }
  }
  __shared__ double red[4][4 * NPT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 2 * NPT; ++j) {
    double a = accK[j], b = accH[j];
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      red[warp][j] = a;
      red[warp][2 * NPT + j] = b;
    }
  }
  __syncthreads();
  if (threadIdx.x < NPT) {
    const int j = threadIdx.x;
    double kr = 0, ki = 0, hr = 0, hi2 = 0;
    for (int wv = 0; wv < 4; ++wv) {
      kr += red[wv][2 * j];
      ki += red[wv][2 * j + 1];
      hr += red[wv][2 * NPT + 2 * j];
      hi2 += red[wv][2 * NPT + 2 * j + 1];
    }
    if (self) {
      // PV int_0^h L_j(s) / (s_x - s) ds = L_j(s_x) log(s_x / (h - s_x)) + int_0^h (L_j(s) - L_j(s_x)) / (s_x - s) ds
      auto lag = [&](double s) {
        const double tt = 2.0 * s / h - 1.0;
        double v = 1.0;
        for (int l = 0; l < NPT; ++l)
          if (l != j) v *= tt - c_tnode[l];
        return v / c_lagden[j];
      };
      const double sx = sstar, lx = lag(sx);
      double pv = lx * log(sx / (h - sx));
      for (int g = 0; g < NGL; ++g) {
        const double sgp = 0.5 * h * (c_glx[g] + 1.0);
        pv += 0.5 * h * c_glw[g] * (lag(sgp) - lx) / (sx - sgp);
      }
      hr += sg * (-inv2pi) * pv;
    }
    const long long o = (long long)i * nb + q * NPT + j;
    Kp[o] = make_double2(kr, ki);
    H[o] = make_double2(hr, hi2);
  }
}

// S, Dl in place: Dl += alpha T, S += alpha (K' + I/2), alpha = i eta / k, with
// T[i][j] = sgn_p (2/h) sum_l H[i][p NPT + l] L_jl'(t_l) + k^2 (n_i . n_j) S[i][j]
// (p the panel of node j, jl its index there).
__global__ void k_bie_combine(const double* __restrict__ nx, const double* __restrict__ ny,
                              const double* __restrict__ tx, const double* __restrict__ ty,
                              const double* __restrict__ pnx, const double* __restrict__ pny, int nb, double h,
                              double k, double eta, const double2* __restrict__ Kp, const double2* __restrict__ H,
                              double2* __restrict__ S, double2* __restrict__ Dl) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nb * nb) return;
  const int i = (int)(e / nb), j = (int)(e % nb);
  const int p = j / NPT, jl = j % NPT;
  const double2* hrow = H + (long long)i * nb + (long long)p * NPT;
  double2 t = make_double2(0.0, 0.0);
#pragma unroll
  for (int l = 0; l < NPT; ++l) t = t + c_dref[l * NPT + jl] * hrow[l];
  t = t * (ccw_sign(tx[p], ty[p], pnx[p], pny[p]) * 2.0 / h);
  const double2 sv = S[e];
  t = t + (k * k * (nx[i] * nx[j] + ny[i] * ny[j])) * sv;
  double2 kp = Kp[e];
  if (i == j) kp.x += 0.5;
  const double a = eta / k;  // alpha = i a
  Dl[e] = Dl[e] + make_double2(-a * t.y, a * t.x);
  S[e] = sv + make_double2(-a * kp.y, a * kp.x);
}

void bie_combined(cudaStream_t s, const Boundary& B, double k, double eta, double2* S, double2* Dl, double2* Kp,
                  double2* H) {
  const long long n = (long long)B.nb * B.nb;
  const unsigned g = (unsigned)((n + 255) / 256);
  k_bie_plain_nt<<<g, 256, 0, s>>>(B.x, B.y, B.nx, B.ny, B.w, B.panel, B.tx, B.ty, B.pnx, B.pny, B.nb, k, Kp, H);
  HS_COUNT_LAUNCH();
  k_bie_near_nt<<<dim3(B.nb, NEAR), 128, 0, s>>>(B.x, B.y, B.nx, B.ny, B.panel, B.p0x, B.p0y, B.tx, B.ty, B.pnx,
                                                 B.pny, B.near, B.h, k, B.nb, Kp, H);
  HS_COUNT_LAUNCH();
  k_bie_combine<<<g, 256, 0, s>>>(B.nx, B.ny, B.tx, B.ty, B.pnx, B.pny, B.nb, B.h, k, eta, Kp, H, S, Dl);
  HS_COUNT_LAUNCH();
}

// Dm = D - I/2 (in place), B1 = Dm/(2 i eta) - S/2, B2 = Dm/(2 i eta) + S/2.
__global__ void k_root_ops(int nb, double eta, const double2* __restrict__ S, double2* __restrict__ Dm,
                           double2* __restrict__ B1, double2* __restrict__ B2) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nb * nb) return;
  int i = (int)(e / nb), j = (int)(e % nb);
  double2 d = Dm[e];
  if (i == j) d.x -= 0.5;
  Dm[e] = d;
  // d / (2 i eta) = -i d / (2 eta)
  double2 q = make_double2(d.y / (2.0 * eta), -d.x / (2.0 * eta));
  double2 sh = make_double2(0.5 * S[e].x, 0.5 * S[e].y);
  B1[e] = q - sh;
  B2[e] = q + sh;
}

void bie_root_ops(cudaStream_t s, int nb, double eta, const double2* S, double2* Dm, double2* B1, double2* B2) {
  long long n = (long long)nb * nb;
  k_root_ops<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(nb, eta, S, Dm, B1, B2);
  HS_COUNT_LAUNCH();
}

__global__ void k_incident_plane(const double* __restrict__ x, const double* __restrict__ y,
                                 const double* __restrict__ nx, const double* __restrict__ ny, int nb, double k,
                                 const double* __restrict__ alphas, int M, double2* __restrict__ ui,
                                 double2* __restrict__ dni) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nb * M) return;
  int j = (int)(e / M), m = (int)(e % M);
  double ca, sa;
  sincos(alphas[m], &sa, &ca);
  double ph = k * (x[j] * ca + y[j] * sa);
  double c, sn;
  sincos(ph, &sn, &c);
  double dn = k * (nx[j] * ca + ny[j] * sa);
  ui[e] = make_double2(c, sn);
  dni[e] = make_double2(-dn * sn, dn * c);  // i k (n.d) e^{i ph}
}

void incident_plane(cudaStream_t s, const Boundary& B, double k, const double* alphas, int M, double2* ui,
                    double2* dni) {
  long long n = (long long)B.nb * M;
  k_incident_plane<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(B.x, B.y, B.nx, B.ny, B.nb, k, alphas, M, ui, dni);
  HS_COUNT_LAUNCH();
}

// A2[p][j] = dG/dn_y(x_p, y_j) w_j  (j < nb),  -G(x_p, y_{j-nb}) w  (j >= nb).
__global__ void k_farfield_matrix(const double* __restrict__ x, const double* __restrict__ y,
                                  const double* __restrict__ nx, const double* __restrict__ ny,
                                  const double* __restrict__ w, int nb, double k, double R,
                                  const double* __restrict__ thetas, int P, double2* __restrict__ A2) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)P * 2 * nb) return;
  int p = (int)(e / (2 * nb)), jj = (int)(e % (2 * nb));
  int j = jj < nb ? jj : jj - nb;
  double ct, st;
  sincos(thetas[p], &st, &ct);
  double dx = R * ct - x[j], dy = R * st - y[j];
  double r = sqrt(dx * dx + dy * dy);
  double2 v;
  if (jj < nb) {
    v = dg_kernel(k * r, k, (dx * nx[j] + dy * ny[j]) / r);
  } else {
    v = -g_kernel(k * r);
  }
  A2[e] = make_double2(v.x * w[j], v.y * w[j]);
}

void farfield_matrix(cudaStream_t s, const Boundary& B, double k, double R, const double* thetas, int P,
                     double2* A2) {
  long long n = (long long)P * 2 * B.nb;
  k_farfield_matrix<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(B.x, B.y, B.nx, B.ny, B.w, B.nb, k, R, thetas, P, A2);
  HS_COUNT_LAUNCH();
}

// Scattered boundary data from the root impedances: u = (f - g)/(2 i eta),
// d_n u = (f + g)/2, minus the incident traces.  PS = [phi_s; psi_s] (2 nb x M).
__global__ void k_boundary_data(int nb, int M, double eta, const double2* __restrict__ f,
                                const double2* __restrict__ g, const double2* __restrict__ ui,
                                const double2* __restrict__ dni, double2* __restrict__ PS) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nb * M) return;
  double2 a = f[e] - g[e], b = f[e] + g[e];
  // (a)/(2 i eta) = -i a / (2 eta)
  double2 phi = make_double2(a.y / (2.0 * eta), -a.x / (2.0 * eta)) - ui[e];
  double2 psi = make_double2(0.5 * b.x, 0.5 * b.y) - dni[e];
  PS[e] = phi;
  PS[(long long)nb * M + e] = psi;
}

void boundary_data(cudaStream_t s, int nb, int M, double eta, const double2* f, const double2* g, const double2* ui,
                   const double2* dni, double2* PS) {
  long long n = (long long)nb * M;
  k_boundary_data<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(nb, M, eta, f, g, ui, dni, PS);
  HS_COUNT_LAUNCH();
}

// Adjoint of the receiver functional at the root: with a = A2[:, :nb]^T and
// b = A2[:, nb:]^T,  E = -a/(2 i eta) + b/2,  CP = a/(2 i eta) + b/2.
__global__ void k_adjoint_root_init(int nb, int P, double eta, const double2* __restrict__ A2,
                                    double2* __restrict__ E, double2* __restrict__ CP) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nb * P) return;
  int j = (int)(e / P), p = (int)(e % P);
  double2 a = A2[(long long)p * 2 * nb + j], b = A2[(long long)p * 2 * nb + nb + j];
  double2 ai = make_double2(a.y / (2.0 * eta), -a.x / (2.0 * eta));  // a / (2 i eta)
  double2 bh = make_double2(0.5 * b.x, 0.5 * b.y);
  E[e] = bh - ai;
  CP[e] = bh + ai;
}

void adjoint_root_init(cudaStream_t s, int nb, int P, double eta, const double2* A2, double2* E, double2* CP) {
  long long n = (long long)nb * P;
  k_adjoint_root_init<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(nb, P, eta, A2, E, CP);
  HS_COUNT_LAUNCH();
}

}  // namespace hs
