// Quadtree of the direct solver (Sec. 2): leaf sizes, merge levels and the
// device routines that build and sweep it.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"
#include "linalg.cuh"

namespace hs {

constexpr int NI = 196;  // interior nodes of a 16 x 16 leaf
constexpr int NE = 56;   // non-corner edge nodes (boundary data of a leaf)
constexpr int NL = 252;  // NI + NE: the leaf's unknowns

struct LeafScratch {  // per-chunk scratch of the leaf build
  double *Aii, *Aie, *Ni, *NiT, *Ne;
  double2 *K, *Kinv;
  int *piv, *pivK;
};

// One level of merges: pairs of child boxes (sx x sy leaves each) merged
// horizontally (west-east) or vertically (south-north) into nbox parents.
struct Level {
  int horiz, sx, sy;
  int nc, ni, np;  // child boundary size, interface size, parent boundary size
  int nbox;
  int *d_alpha, *d_beta;       // child box ids of each parent
  int *d_src;                  // parent boundary node -> (child << 20) | child-local index
  int *d_I3a, *d_I3b;          // interface nodes in the alpha / beta child
  double2 *XZ;                 // [nbox][2 ni][np]  interface impedances from the parent's
  double2 *U2;                 // [nbox][np][2 ni]  interface -> parent outgoing impedance
  double2 *A33, *B33, *M;      // [nbox][ni][ni]; M holds the LU of I - B33 A33
  int *Mpiv;                   // [nbox][ni]
  double2 *R;                  // [nbox][np][np]  parent impedance-to-impedance maps
};

void upload_cheb_diff(const double* D1, cudaStream_t s);
void sine_eval_grid(cudaStream_t s, const double* c, int S1, int S2, const double* xg, int nL, double* sx,
                    double* sy, double* T, double* Qg, double* q, int* bad);
void check_q(cudaStream_t s, const double* q, long long n, int* bad);
void leaf_build_chunk(cudaStream_t s, const double* q, int leaf0, int nleaf, double k, double h, LeafScratch& w,
                      double2* R, double2* Y, double2* Q, int* info);

void merge_level(cudaStream_t s, const Level& L, const double2* Rc, int* info);
void sweep_down_level(cudaStream_t s, const Level& L, const double2* Fp, double2* T3, double2* Fc, int nrhs);
void sweep_adjoint_level(cudaStream_t s, const Level& L, const double2* Lp, double2* MU, double2* Lc, int nrhs);

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
                           cudaStream_t s);
void bie_matrices(cudaStream_t s, const Boundary& B, double k, double2* S, double2* Dl);
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
void contract_jacobian(cudaStream_t s, const double2* Ug, const double2* Zg, int M, int P, int nX, const double* sx,
                       const double* sy, int S1, int S2, double k2, double2* J);
void split_stack(cudaStream_t s, const double2* J, int rows, int cols, double* Jst);
void residual(cudaStream_t s, const double* data, const double2* F, int n, double2* res, double* rst, double* out2);
void add_lambda(cudaStream_t s, double* A, int n, double lambda_rel);
void gradient_combine(cudaStream_t s, const double2* Ug, const double2* Zmix, int M, long long npts, double* hre);
void conj_neg(cudaStream_t s, double2* v, int n);
void half_in_place(cudaStream_t s, double* v);

}  // namespace hs
