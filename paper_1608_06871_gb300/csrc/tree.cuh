// Quadtree of the direct solver (Sec. 2): leaf sizes, merge levels and the
// device routines that build and sweep it, in FP64 (double2 operators) or
// FP32 (float2 operators, the mixed-precision path).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"
#include "linalg.cuh"

namespace hs {

constexpr int NI = 196;  // interior nodes of a 16 x 16 leaf
constexpr int NE = 56;   // non-corner edge nodes (boundary data of a leaf)
constexpr int NL = 252;  // NI + NE: the leaf's unknowns

template <typename T> struct LeafScratchT {  // leaf build scratch; in the mixed path it is kept (refinement)
  using C = typename prec<T>::C;
  T *Aii, *Aie, *Ni, *NiT, *Ne;   // Aii holds the LU factors, Aie holds X = Aii^{-1} Aie afterwards
  C *K, *Kinv;
  int *piv, *pivK;
  T* Ainv = nullptr;  // mixed path: Aii^{-1} explicitly (the particular solves apply it with one GEMM)
  // impedance form: the 252 x 252 leaf system, L^{-T} [0; I] (FP64 adjoint operator Q), and
  // the particular-solution operator P = L^{-1} [I; 0] (mixed path: refinement body loads)
  C *L = nullptr, *Et = nullptr, *P = nullptr;
  int* pivL = nullptr;
};
using LeafScratch = LeafScratchT<double>;

// Index maps of one level of merges: pairs of child boxes (sx x sy leaves
// each) merged horizontally (west-east) or vertically (south-north).
struct LevelMaps {
  int horiz, sx, sy;
  int nc, ni, np;              // child boundary size, interface size, parent boundary size
  int n1;                      // parent nodes from alpha: the parent order is [alpha exterior; beta exterior]
  int nbox, nbx_p;             // parent boxes, parents per row
  int *d_alpha, *d_beta;       // child box ids of each parent
  int *d_src;                  // parent boundary node -> (child << 20) | child-local index
  int *d_I3a, *d_I3b;          // interface nodes in the alpha / beta child
};

// Operators stored per level for the sweeps (C = double2 or float2).
// Parent boundary nodes are ordered [alpha exterior; beta exterior], so the
// parent map update R = blockdiag(A11, B22) + [A13 X; B23 Z] is two dense GEMMs.
template <typename C> struct LevelOps {
  C* XZ;      // [nbox][2 ni][np]  interface impedances from the parent's: [X; Z]
  C* U2;      // [nbox][np][ni]  rows < n1: A13 (alpha exterior x interface), rows >= n1: B23
  C *A33, *B33, *M;  // [nbox][ni][ni]; M: LU of I - B33 A33 (FP64), W = (I - B33 A33)^{-1} (FP32)
  int* Mpiv;  // [nbox][ni]
  C* R;       // [nbox][np][np]  parent impedance-to-impedance maps
};

// Legacy FP64 view used by the FP64 path.
struct Level : LevelMaps, LevelOps<double2> {};

void upload_cheb_diff(const double* D1, cudaStream_t s);
void sine_eval_grid(cudaStream_t s, const double* c, int S1, int S2, const double* xg, int nL, double* sx,
                    double* sy, double* T, double* Qg, double* q, int* bad);
void check_q(cudaStream_t s, const double* q, long long n, int* bad);
// k: the wavenumber on the host (GEMM scalars), d_k: the same on the device (read
// by the kernels, so that a captured build serves every k).
template <typename T>
void leaf_build_chunk(cudaStream_t s, const double* q, int leaf0, int nleaf, double k, const double* d_k, double h,
                      LeafScratchT<T>& w, typename prec<T>::C* R, typename prec<T>::C* Y, typename prec<T>::C* Q,
                      int* info);
// The same outputs (R, Y, and Q when non-NULL, with w.Et) from the impedance form of the
// leaf problem (needs w.L, w.pivL): one LU of the 252 x 252 complex system with the incoming
// impedance on the edge, solvable where A_ii is singular (the leaf's Dirichlet eigenvalues);
// with w.P also the particular-solution operator L^{-1} [I; 0] for the chunk's leaves.
template <typename T>
void leaf_build_chunk_impedance(cudaStream_t s, const double* q, int leaf0, int nleaf, double k, const double* d_k,
                                double h, LeafScratchT<T>& w, typename prec<T>::C* R, typename prec<T>::C* Y,
                                typename prec<T>::C* Q, int* info);

template <typename C> void merge_level(cudaStream_t s, const LevelMaps& L, const LevelOps<C>& O, const C* Rc, int* info);
// Downward sweep of one level.  If t3_loaded, T3 already holds the particular
// interface impedances [t_a; t_b] of the upward pass and is added to.
template <typename C>
void sweep_down_level(cudaStream_t s, const LevelMaps& L, const LevelOps<C>& O, const C* Fp, C* T3, C* Fc, int nrhs,
                      bool t3_loaded);
// Transposed downward sweep of one level (the adjoint of sweep_up_level's map
// from the children's particular impedances and the interface terms to the
// parent's): parent loads Lp give the children's Lc; MU ([nbox][2 ni][nrhs])
// ends as [Wt; la3], whose halves are the adjoints of s_a (Wt) and of s_b
// (-la3).  With mu_loaded, MU holds on entry the adjoint of the particular
// interface impedances [t_a; t_b] (from sweep_adjoint_up_level) and is added to.
template <typename C>
void sweep_adjoint_level(cudaStream_t s, const LevelMaps& L, const LevelOps<C>& O, const C* Lp, C* MU, C* Lc,
                         int nrhs, bool w_explicit = false, bool mu_loaded = false);
// Transposed upward sweep of one level (the adjoint of sweep_down_level):
// children's adjoint loads Lc give the parent's Lp and the adjoint of the
// interface impedances MU = [Lc_alpha(I3a); Lc_beta(I3b)] ([nbox][2 ni][nrhs]).
template <typename C>
void sweep_adjoint_up_level(cudaStream_t s, const LevelMaps& L, const LevelOps<C>& O, const C* Lc, C* MU, C* Lp,
                            int nrhs);
// Upward (particular) pass of one level: children's outgoing particular
// impedances Hc and the interface residual terms S3 ([s_a; s_b] per box) give
// the particular interface impedances TT = [t_a; t_b] (kept for the downward
// pass) and the parent's particular impedances Hp.  S3 is consumed (reused as
// scratch).  For C = float2 the level's M holds W = (I - B33 A33)^{-1} itself
// (merge_level stores it explicitly), for C = double2 its LU factors.
template <typename C>
void sweep_up_level(cudaStream_t s, const LevelMaps& L, const LevelOps<C>& O, const C* Hc, C* S3, C* TT, C* Hp,
                    int nrhs);

// Compatibility wrappers for the FP64 path.
inline void merge_level(cudaStream_t s, const Level& L, const double2* Rc, int* info) {
  merge_level<double2>(s, L, L, Rc, info);
}
inline void sweep_down_level(cudaStream_t s, const Level& L, const double2* Fp, double2* T3, double2* Fc, int nrhs) {
  sweep_down_level<double2>(s, L, L, Fp, T3, Fc, nrhs, false);
}
inline void sweep_adjoint_level(cudaStream_t s, const Level& L, const double2* Lp, double2* MU, double2* Lc, int nrhs) {
  sweep_adjoint_level<double2>(s, L, L, Lp, MU, Lc, nrhs);
}

// Boundary integral part (bie.cu)
struct Boundary {
  int nb;              // boundary nodes
  int npanel;
  double h;
  double *x, *y, *nx, *ny, *w;  // node coordinates, outward normals, ds weights
  int *panel;                   // panel of each node
  double *p0x, *p0y, *tx, *ty, *pnx, *pny;  // panel start, tangent, normal
  int *near;                    // [npanel][5] near panels (-1 padded)
};
void upload_quad_constants(const double* gl_x, const double* gl_w, const double* tnodes, const double* lagden,
                           const double* dref, cudaStream_t s);
void bie_matrices(cudaStream_t s, const Boundary& B, double k, double2* S, double2* Dl);
// Burton-Miller rows in place: Dl += alpha T, S += alpha (K' + I/2), alpha = i eta / k
// (Kp, H: nb x nb scratch for K' and the tangential derivative of S).
void bie_combined(cudaStream_t s, const Boundary& B, double k, double eta, double2* S, double2* Dl, double2* Kp,
                  double2* H);
void bie_root_ops(cudaStream_t s, int nb, double eta, const double2* S, double2* Dm, double2* B1, double2* B2);
void incident_plane(cudaStream_t s, const Boundary& B, double k, const double* alphas, int M, double2* ui,
                    double2* dni);
void farfield_matrix(cudaStream_t s, const Boundary& B, double k, double R, const double* thetas, int P, double2* A2);
void boundary_data(cudaStream_t s, int nb, int M, double eta, const double2* f, const double2* g, const double2* ui,
                   const double2* dni, double2* PS);
void adjoint_root_init(cudaStream_t s, int nb, int P, double eta, const double2* A2, double2* E, double2* CP);

// Jacobian, gradient and Gauss-Newton pieces (jac.cu)
void leaf_to_grid(cudaStream_t s, const double2* Uleaf, int nrows_leaf, int nL, int nrhs, double2* G);
void leaf_to_nodes(cudaStream_t s, const double2* Uleaf, int nL, int nrhs, double2* out);
void interior_sine_tables(cudaStream_t s, const double* xg_int, int n, int S1, int S2, double* sx, double* sy);
// Pairs per chunk of the contraction within budget_bytes of W and T (the
// emulated FP64 product needs contract_emulated_bytes on top).
int contract_chunk(int M, int P, int nX, int S1, size_t budget_bytes);
size_t contract_emulated_bytes(int C, int nX, int S1, int S2);
// scratch: emulated-product slices (contract_emulated_bytes), or NULL for the
// FP64 SIMT GEMMs.
void contract_jacobian(cudaStream_t s, const double2* Ug, const double2* Zg, int M, int P, int nX, const double* sx,
                       const double* sy, int S1, int S2, double k2, double2* J, double2* W, double2* T, int C,
                       void* scratch, size_t scratch_bytes);
void split_stack(cudaStream_t s, const double2* J, int rows, int cols, double* Jst);
// J v and Re(J^H f) from the forward and adjoint fields on the interior grid (no J formed).
void apply_J(cudaStream_t s, const double2* Ug, const double2* Zg, int M, int P, int nX, const double* sx,
             const double* sy, int S1, int S2, double k2, const double* v, double* G1, double* qv, double2* Y,
             double2* y);
void apply_JH(cudaStream_t s, const double2* Ug, const double2* Zg, int M, int P, int nX, const double* sx,
              const double* sy, int S1, int S2, double k2, const double2* f, double2* fc, double2* Zmix, double* h,
              double* T1, double* g);
// Explicit complex FP32 Jacobian (W: C nX^2, T: C nX S1 values; sxc: nX S1, sy32:
// nX S2; C from contract_chunk32), and its products with FP64 sums: y = J v
// (rows complex outputs, real v) and g = Re(J^H u) (part: gemvT_parts(rows) * n
// doubles).
int contract_chunk32(int M, int P, int nX, int S1, size_t budget_bytes);
void contract_jacobian32(cudaStream_t s, const double2* Ug, const double2* Zg, int M, int P, int nX, const double* sx,
                         const double* sy, int S1, int S2, double k2, float2* J, float2* sxc, float* sy32, float2* W,
                         float2* T, int C);
int gemvT_parts(long long rows);
void gemv32(cudaStream_t s, const float2* J, long long rows, int n, const double* v, double2* y);
void gemvT32(cudaStream_t s, const float2* J, long long rows, int n, const double2* u, double* part, double* g);
// The same on an explicit FP64 Jacobian.
void gemv64(cudaStream_t s, const double2* J, long long rows, int n, const double* v, double2* y);
void gemvT64(cudaStream_t s, const double2* J, long long rows, int n, const double2* u, double* part, double* g);
// A = Jst^T Jst (n x n) by block rows of its lower part, mirrored.
void normal_matrix(cudaStream_t s, const double* Jst, int rows, int n, double* A);
// The same from the transposed stack JstT = [Re J; Im J]^T (n x 2 MP, written by
// split_stack_t) with the emulated FP64 product; false if it could not run.
void split_stack_t(cudaStream_t s, const double2* J, int rows, int cols, double* JstT);
size_t normal_matrix_emulated_bytes(int rows, int n);
bool normal_matrix_emulated(cudaStream_t s, double* JstT, int rows, int n, double* A, void* scratch, size_t bytes);
void residual(cudaStream_t s, const double* data, const double2* F, int n, double2* res, double* rst, double* out2);
void add_lambda(cudaStream_t s, double* A, int n, double lambda_rel);
void gradient_combine(cudaStream_t s, const double2* Ug, const double2* Zmix, int M, long long npts, double* hre);
void conj_neg(cudaStream_t s, double2* v, int n);
void half_in_place(cudaStream_t s, double* v);

// Mixed-precision refinement pieces (refine.cu)
void convert_d2f(cudaStream_t s, const double2* a, float2* b, long long n);
void convert_f2d_add(cudaStream_t s, const float2* a, double2* b, long long n);  // b += a
// D1: device copy of the 16 x 16 Chebyshev-Lobatto differentiation matrix on [-1, 1].
void residual_pde(cudaStream_t s, const double2* X, const double* q, const double* D1, int nleaf, double k, double h,
                  int nrhs, float2* RP);
void residual_iface(cudaStream_t s, const LevelMaps& L, const double2* X, const double* D1, int nL, double h,
                    const double* d_k, int nrhs, float2* S3);
void boundary_gather(cudaStream_t s, const double2* X, const double* D1, int nL, double h, int nrhs, double2* ub,
                     double2* psib);
void leaf_particular(cudaStream_t s, const LeafScratchT<float>& w, int nleaf, const double* d_k, int nrhs, float2* Upart,
                     float2* H, float2* tmp, float2* wtmp);
void scattered_data(cudaStream_t s, const double2* ub, const double2* psib, const double2* ui, const double2* dni,
                    long long n, double2* PS);
// FP32 scattered boundary data [u (- u_inc); d_n u (- d_n u_inc)] of an FP32 leaf field, and out += |a|^2.
void scattered32(cudaStream_t s, const float2* U32, const double* D1, int nL, double h, int nrhs, const double2* ui,
                 const double2* dni, bool sub_inc, float2* PS);
void norm2_32(cudaStream_t s, const float2* a, long long n, double* out);
// Adjoint refinement (refine.cu): G (FP32, leaf layout [leaf][252][nrhs]) =
// L - A^T Y in FP64 for the adjoint Y (Ypde [leaf][196][nrhs]; Yif, every
// merge level's [nbox][2 ni][nrhs] adjoints of (s_a, s_b) back to back; V =
// [D - I/2, -S]^T Yext, [2 nb][nrhs], or NULL when Yext = 0), L the receiver
// functionals from A2 ([nrhs][2 nb]).  desc[leaf][56] = (x, y, kind): kind 2 =
// boundary node x; kind 0 / 1 = alpha / beta side of the interface row whose s_a
// adjoint is at Yif[x * nrhs], s_b at Yif[(x + y) * nrhs].  first: Y = 0.
void adjoint_residual(cudaStream_t s, const double2* Ypde, const int4* desc, const double2* Yif, const double2* A2,
                      const double2* V, const double* q, const double* D1, int nleaf, int nb, double k, double h,
                      double eta, int nrhs, bool first, float2* G);
// G edge rows += -2 i eta H  (H [leaf][56][nrhs]).
void leaf_hadj(cudaStream_t s, const float2* H, int nleaf, double eta, int nrhs, float2* G);
// Y += [MU top; -MU bottom] per box (one level, [nbox][2 ni][nrhs]).
void iface_adj_add(cudaStream_t s, const float2* MU, int nbox, int ni, int nrhs, double2* Y);
// DS = [D - I/2, -S] (nb x 2 nb) in FP64 and FP32.
void stack_exterior(cudaStream_t s, const double2* Dm, const double2* S, int nb, double2* DS, float2* DS32);
// dst[r][:] = src[idx[r]][:] (rows of ncols elements); dst[a][b] = src[idx[a]][idx[b]] for square matrices.
template <typename C> void permute_rows(cudaStream_t s, const C* src, const int* idx, int nrows, int ncols, C* dst);
template <typename C> void permute_square(cudaStream_t s, const C* src, const int* idx, int n, C* dst);

}  // namespace hs
