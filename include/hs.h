/*
 * hs.h -- C ABI of libhs: the hot path of recursive linearization for 2-D
 * inverse scattering (Borges, Gillman, Greengard, arXiv 1608.06871) at one
 * frequency k, on one GPU.
 *
 * Problem (paper Sec. 1, eqs. origpde, srad, farfielddef): a contrast q(x)
 * supported in Omega = [-1, 1]^2, the total field u = u_inc + u_s with
 *     Lap u + k^2 (1 - q) u = 0,   u_inc = exp(i k x.d),   u_s radiating,
 * and the measured data u_far(theta) = u_s(R cos theta, R sin theta).
 * The contrast is the truncated sine series of Sec. 3.2 (eq. sineseries) on
 * [-1,1]^2:  q(x) = sum_{m1=1..S1, m2=1..S2} c[m1-1][m2-1] s_m1(x1) s_m2(x2),
 * s_m(t) = sin(m pi (t + 1) / 2).
 *
 * Discretisation: n_L x n_L leaves of 16 x 16 Chebyshev-Lobatto points (Sec. 2,
 * Table 1), interior solved by hierarchical merges of impedance-to-impedance
 * maps (Sec. 2), exterior by the Green identity (D - I/2) u_s = S d_n u_s on
 * the boundary of Omega (Sec. 2, Remark).
 *
 * Conventions for every call:
 *  - Arrays are owned by the caller.  Plain pointers (no suffix) are HOST
 *    memory; calls ending in _dev take DEVICE pointers and a cudaStream_t
 *    passed as void* (NULL = the context's stream; pass cudaStreamLegacy,
 *    (void*)1, for the legacy default stream) and return without
 *    synchronising that stream.
 *  - Complex arrays are interleaved (re, im) doubles, row-major.
 *  - Return value: HS_OK (0) or a negative HS_E* code; hs_last_error()
 *    then gives a one-line reason.  No call aborts, traps or prints.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef HS_H
#define HS_H

#ifdef __cplusplus
extern "C" {
#endif

#define HS_OK 0
#define HS_EINVAL (-1)      /* bad size, NaN, or 1 - q <= 0 on the grid      */
#define HS_ENOTBUILT (-2)   /* solve/jacobian before hs_build                 */
#define HS_ENOMEM (-3)      /* device allocation failed                       */
#define HS_ECUDA (-4)       /* CUDA runtime error                             */
#define HS_ESINGULAR (-5)   /* zero pivot in a factorisation                  */
#define HS_ENOCONV (-6)     /* iterative refinement did not converge          */
#define HS_ETIMEOUT (-7)    /* a bounded device wait gave up                  */

#define HS_FP64 0   /* every step in complex FP64                            */
#define HS_MIXED 1  /* FP32 factors and sweep, FP64 residual refinement       */

typedef struct hs_ctx hs_ctx;

typedef struct hs_config {
  double R;             /* receiver circle radius (> sqrt(2)); 3.0 in the workloads */
  int leaves_per_side;  /* n_L, a power of two, 1..256                              */
  int S1, S2;           /* sine modes per axis (1..512)                             */
  int precision;        /* HS_FP64 or HS_MIXED                                      */
  int device;           /* CUDA device ordinal                                      */
  void* stream;         /* cudaStream_t for all work, or NULL for a private stream  */
  double refine_tol;    /* HS_MIXED: stop when the estimated relative error of the
                           far field (last update x rho/(1-rho), rho the observed
                           contraction per pass) is below this (default 1e-9)       */
  int refine_max_iter;  /* HS_MIXED: maximum refinement sweeps (default 8 if <= 0)  */
  double bm_eta;        /* exterior rows on the boundary (Sec. 2, Remark): 0 = Green's
                           identity (D - I/2) u_s = S d_n u_s, singular where k^2 is a
                           Dirichlet eigenvalue of the square; > 0 = its Burton-Miller
                           combination with the normal-derivative identity
                           T u_s = (K' + I/2) d_n u_s, coupling i bm_eta / k, solvable
                           at every k (1 is the usual choice); < 0 or NaN: HS_EINVAL */
  int leaf_impedance;   /* leaf elimination (Sec. 2, HPS leaves): 0 = through the
                           Dirichlet block A_ii (needs k sqrt(1-q) h away from the
                           leaf's Dirichlet eigenvalues pi sqrt(a^2+b^2)); 1 = one
                           LU of the leaf's impedance system (incoming impedance on
                           the edge), solvable at every k h (HS_MIXED contexts keep
                           its particular-solution operator for the refinement:
                           0.4 MB per leaf more); other values: HS_EINVAL */
} hs_config;

/* Create a context on cfg->device (copies cfg).  Allocates nothing large until
 * hs_build.  Errors: HS_EINVAL on bad sizes, HS_ECUDA if the device is absent. */
int hs_create(hs_ctx** out, const hs_config* cfg);

/* Factor the discrete operator for the contrast given by sine coefficients
 * c (host, S1*S2 doubles, c[(m1-1)*S2 + (m2-1)]) at wavenumber k > 0
 * (Sec. 3.2 eq. sineseries for q; Sec. 2 for the factorisation, which the
 * paper performs once per Newton step, Sec. 3.3).  Evaluates q on every leaf
 * node on the GPU.  Errors: HS_EINVAL (NaN, k <= 0, shape mismatch,
 * 1 - q <= 0 at a node), HS_ESINGULAR, HS_ENOMEM, HS_ECUDA. */
int hs_build(hs_ctx* ctx, const double* c, int S1, int S2, double k);

/* As hs_build, but q is given directly at the leaf nodes (host array of
 * n_L*n_L*256 doubles in the order of hs_node_coords).  Used to generate
 * measured data from a contrast that is not a sine series. */
int hs_build_nodes(hs_ctx* ctx, const double* q_nodes, double k);

/* Leaf node coordinates (host arrays of n_L*n_L*256 doubles): node index
 * ((iy*n_L + ix)*16 + a)*16 + b is the point (x_a, y_b) of leaf (ix, iy). */
int hs_node_coords(const hs_ctx* ctx, double* x, double* y);

/* Forward solves (Sec. 1 eq. farfielddef; Sec. 3 eq. singfreqsys): for each
 * incidence angle alpha_m (d = (cos, sin)) and receiver angle theta_p, the
 * scattered field at R (cos theta_p, sin theta_p).  Output ufar: M x P
 * complex, row-major (m slow).  Requires hs_build. */
int hs_solve(hs_ctx* ctx, const double* alphas, int M, const double* thetas, int P,
             double* ufar);
int hs_solve_dev(hs_ctx* ctx, const double* alphas, int M, const double* thetas, int P,
                 double* ufar, void* stream);

/* Far-field solve that allocates no device memory (the paper has no
 * counterpart).  For callers that must not allocate at call time: code whose
 * device memory belongs to another allocator (a framework's caching pool, or
 * a fixed arena sized at start-up), where an allocation made behind its back
 * would break its accounting or fail under its memory cap.  Same arguments
 * and results as hs_solve_dev (device pointers); the factors come from
 * hs_build on ctx, which must have been called before, on an HS_FP64 context
 * (HS_EINVAL otherwise: the mixed path's refinement needs far more scratch).
 * Scratch: one 16 MiB static device array compiled into libhs (every GPU
 * that loads the library holds it until the process exits).  The call needs
 * 16 * N_b * (6 M + 2 P) bytes of it, N_b = 56 n_L; larger M, P are rejected
 * with HS_EINVAL.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current and keeps it for
 * the life of the process; make that first call before any stream capture.
 * A cudaDeviceReset (or anything else that destroys the device's primary
 * context) invalidates the kept address: after one, do not call this
 * function again in that process.  All calls share the array and it keeps
 * the last call's contents (every region is written before it is read, so
 * nothing needs clearing): calls whose GPU work overlaps -- on different
 * streams or from different contexts -- race on it; serialise them. */
int hs_solve_noalloc(hs_ctx* ctx, const double* alphas, int M, const double* thetas, int P,
                     double* ufar, void* stream);

/* Full forward solve (Sec. 2: one right-hand side per incidence, pushed down
 * the tree to every leaf node; Sec. 1 eq. farfielddef for the data): the far
 * field ufar (M x P complex, as hs_solve) and the total field u on every leaf
 * node (M x n_L*n_L*256 complex, node order of hs_node_coords, corners 0), both
 * device pointers.  With HS_MIXED one refinement run yields both. */
int hs_forward_dev(hs_ctx* ctx, const double* alphas, int M, const double* thetas, int P, double* ufar,
                   double* u, void* stream);

/* Total fields on the leaf nodes for M plane-wave incidences (device output,
 * M x n_L*n_L*256 complex, node order of hs_node_coords; corner nodes of
 * each leaf are not part of the discretisation and are set to 0). */
int hs_fields_dev(hs_ctx* ctx, const double* alphas, int M, double* u, void* stream);

/* Jacobian of the data with respect to the sine coefficients at the built
 * contrast (Theorem 3.1, eqs. Jdef/vdef, read on the basis of eq. sineseries):
 * J[(m*P + p)][(m1-1)*S2 + (m2-1)] = d u_far(m, p) / d c[m1][m2], complex,
 * (M*P) x (S1*S2) row-major.  Assembled by discrete reciprocity (the adjoint
 * of Theorem 3.2): forward fields times adjoint fields, projected onto the
 * sine basis.  On an HS_MIXED context both fields come from FP64 iterative
 * refinement of FP32 solves -- the forward fields as in hs_solve, the adjoint
 * fields by refinement on the transposed system (FP64 residual of every
 * transposed row, FP32 transposed correction solve) -- and the contraction
 * runs in FP64, so J agrees with the FP64 context's to the refinement
 * tolerance.  Errors as hs_solve, plus HS_ENOCONV if the adjoint refinement
 * does not reach refine_tol in refine_max_iter passes. */
int hs_jacobian(hs_ctx* ctx, const double* alphas, int M, const double* thetas, int P,
                double* J);
int hs_jacobian_dev(hs_ctx* ctx, const double* alphas, int M, const double* thetas, int P,
                    double* J, void* stream);

/* One Gauss-Newton step from the normal equations (Sec. 3.3, eq. normaleq)
 * in the real coefficients: with r = data - F(c) and J as above,
 *   (Re(J^H J) + lambda I) dc = Re(J^H r),  lambda = lambda_rel * tr(Re J^H J) / (S1*S2),
 * then c <- c + dc.  c_inout (host, S1*S2) must be the coefficients the
 * context was last built with; on return the context holds the factors of
 * the OLD c (call hs_build again to factor the new one).  data: M x P complex
 * (host).  resid_norm_out (optional): ||r||_2 before the step.  HS_FP64 or
 * HS_MIXED context (on a mixed one F, J and the fields behind them are the
 * refined ones of hs_solve and hs_jacobian; the normal equations are FP64). */
int hs_gn_step(hs_ctx* ctx, const double* data, const double* alphas, int M,
               const double* thetas, int P, double lambda_rel, double* c_inout,
               double* resid_norm_out);

/* One Gauss-Newton step with the linearized least-squares problem solved by
 * LSQR (Paige and Saunders), as the paper's experiments do (Sec. 4: LSQR,
 * algebraically identical to conjugate gradients on eq. normaleq, stopped at a
 * tolerance of 1e-3):  min over real dc of ||J dc - r||^2 + damp^2 ||dc||^2,
 * r = data - F(c), dc restricted to the modes where mask != 0 (mask: S1*S2
 * bytes in the order of c, or NULL for all modes; e.g. the triangle
 * m1 + m2 <= S of Sec. 3.2).  J comes from the forward and adjoint fields of
 * the built contrast (Theorem 3.1 / 3.2).  products: HS_FP64 -- J is formed
 * once in FP64 by the emulated FP64 contraction on the tensor cores and every
 * iteration reads it twice (with the emulation switched off, J and J^H are
 * applied from the fields by two FP64 grid contractions per iteration);
 * HS_MIXED -- J is formed once in complex FP32 and every iteration reads it
 * twice with FP64 sums (for loose tolerances such as the paper's 1e-3); on an HS_MIXED
 * context its adjoint fields get one FP64-residual correction after the FP32
 * solve.  Either way J v
 * and J^H u stay exact transposes of one matrix.  The iteration's vectors live on the
 * host.  Stops when the relative residual or the relative normal-equations
 * residual (LSQR's own estimates) is at most tol, or after max_iter
 * iterations; *iters_out (optional) receives the count.  Otherwise as
 * hs_gn_step (c_inout updated, resid_norm_out = ||r||_2 before the step).
 * On an HS_MIXED context the residual, the forward fields and (for products
 * HS_FP64) the adjoint fields come from the refined solves (FP64 accurate), so
 * with products HS_FP64 the step is the FP64 context's to the refinement
 * tolerance; with products HS_MIXED it carries the FP32 rounding of the
 * tensor-core J on either kind of context.  The explicit J needs M P S1 S2
 * complex doubles of device workspace.  Errors: HS_EINVAL (damp < 0, tol < 0,
 * max_iter < 1, bad products, bad sizes, NULL), HS_ENOTBUILT, HS_ENOMEM,
 * HS_ECUDA, HS_ETIMEOUT, HS_ENOCONV. */
int hs_gn_step_lsqr(hs_ctx* ctx, const double* data, const double* alphas, int M,
                    const double* thetas, int P, const unsigned char* mask, double damp,
                    double tol, int max_iter, int products, double* c_inout,
                    double* resid_norm_out, int* iters_out);

/* Gradient of the misfit 0.5 * ||F(c) - data||^2 with respect to the real sine
 * coefficients, grad = Re(J^H (F(c) - data)) (Theorem 3.2 read on the basis),
 * without forming J: one adjoint sweep over the receivers.  grad: S1*S2 doubles
 * (host); misfit_out (optional): the misfit value.  Requires hs_build.  On an
 * HS_MIXED context the misfit, the forward fields and the adjoint fields come
 * from the refined solves (FP64 accurate; HS_ENOCONV if a refinement stalls). */
int hs_gradient(hs_ctx* ctx, const double* data, const double* alphas, int M,
                const double* thetas, int P, double* grad, double* misfit_out);
int hs_gradient_dev(hs_ctx* ctx, const double* data, const double* alphas, int M,
                    const double* thetas, int P, double* grad, double* misfit_out,
                    void* stream);

/* Number of kernel launches issued by this context since creation (for
 * reporting). */
long long hs_launch_count(const hs_ctx* ctx);

/* Last error message of the context (never NULL). */
const char* hs_last_error(const hs_ctx* ctx);

/* Release every device allocation of the context. */
void hs_destroy(hs_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* HS_H */
