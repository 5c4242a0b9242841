// C ABI of libhs (include/hs.h): host-side orchestration of the direct solver
// of Sec. 2 and of the Jacobian / Gauss-Newton step of Sec. 3 on one GPU.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hs.h"
#include "../../include/hs_diag.h"
#include "tree.cuh"

namespace hs {
thread_local long long* g_launch_counter = nullptr;
bool g_use_graphs = true;  // process-wide switch (hs_set_graphs)
// Scratch of the Jacobian contraction for one chunk of (d, p) pairs (Khatri-Rao
// rows and half-projected rows); process-wide (hs_set_contract_budget).
size_t g_contract_budget = size_t(1) << 30;
bool prof_active(int family);
// Test hook (hs_fail_next_allocs): this many of the next device allocations
// of a context fail on the host with HS_ENOMEM, without calling cudaMalloc.
int g_fail_allocs = 0;
}

using namespace hs;

namespace {

// ---- host-side 1-D rules (definitions, computed in double) ----------------
// Chebyshev-Lobatto points t_a = -cos(pi a / (p-1)), ascending.
std::vector<double> lobatto(int p) {
  std::vector<double> t(p);
  for (int a = 0; a < p; ++a) t[a] = -std::cos(M_PI * a / (p - 1));
  return t;
}

// Derivative of the Lagrange interpolant: D[i][j] = L_j'(t_i), from the
// barycentric weights lambda_j = 1 / prod_{l != j} (t_j - t_l).
std::vector<double> diff_matrix(const std::vector<double>& t) {
  int n = (int)t.size();
  std::vector<double> lam(n), D(n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double p = 1.0;
    for (int l = 0; l < n; ++l)
      if (l != j) p *= (t[j] - t[l]);
    lam[j] = 1.0 / p;
  }
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j)
      if (i != j) {
        D[i * n + j] = (lam[j] / lam[i]) / (t[i] - t[j]);
        s += D[i * n + j];
      }
    D[i * n + i] = -s;
  }
  return D;
}

// Fejer's second rule on the n interior points cos(j pi/(n+1)), j = 1..n:
// w_j = 4 sin(th_j)/(n+1) * sum_{l=1}^{ceil(n/2)} sin((2l-1) th_j)/(2l-1).
// Returned in ascending node order (t = -cos).
std::vector<double> fejer2(int n) {
  std::vector<double> w(n);
  for (int j = 1; j <= n; ++j) {
    double th = M_PI * j / (n + 1), s = 0.0;
    for (int l = 1; l <= (n + 1) / 2; ++l) s += std::sin((2 * l - 1) * th) / (2 * l - 1);
    w[j - 1] = 4.0 * std::sin(th) / (n + 1) * s;
  }
  return w;  // symmetric, so the order of t does not matter
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Bump allocator over the context's workspace.  A request beyond the sized
// capacity returns NULL and sets `over`; every caller checks `over` after its
// requests and before any launch, so a sizing mistake is an error, never an
// out-of-bounds access.
struct Arena {
  char* base = nullptr;
  size_t cap = 0, off = 0;
  bool over = false;
  template <typename T> T* get(size_t n) {
    size_t b = (n * sizeof(T) + 255) & ~size_t(255);
    if (off + b > cap) {
      over = true;
      return nullptr;
    }
    T* p = reinterpret_cast<T*>(base + off);
    off += b;
    return p;
  }
  static size_t bytes(size_t n, size_t elt) { return (n * elt + 255) & ~size_t(255); }
};

}  // namespace

// A captured CUDA graph of a fixed launch sequence and the values its launch
// parameters depend on (buffer base, sizes, frequency).
namespace hs {
struct GraphSlot {
  cudaGraphExec_t exec = nullptr;
  const void* base = nullptr;
  int M = -1, P = -1;
  double k = -1.0;
  long long kernels = 0;
  // the key of the last eager run: a sequence is captured on its second use,
  // after one eager run has sized the products' scratch and measured their shapes
  const void* seen_base = nullptr;
  int seen_M = -1, seen_P = -1;
  double seen_k = -1.0;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
  }
};
}  // namespace hs

struct hs_ctx {
  hs_config cfg{};
  int nL = 0, nleaf = 0, n14 = 0, n16 = 0, chunk = 0;
  double h = 0, k = 0;
  int S1 = 0, S2 = 0;
  bool built = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  long long launches = 0;
  std::vector<void*> allocs;  // persistent allocations
  // geometry
  double *d_xg = nullptr, *d_xint = nullptr;
  double *d_q = nullptr, *d_c = nullptr, *d_sx16 = nullptr, *d_sy16 = nullptr, *d_T = nullptr, *d_Qg = nullptr;
  double *d_sxi = nullptr, *d_syi = nullptr;
  int* d_info = nullptr;
  int ninfo = 0;
  // factors
  double2 *d_Rleaf = nullptr, *d_Y = nullptr, *d_Q = nullptr;
  LeafScratch ws{};
  std::vector<Level> levels;
  Boundary B{};
  double2 *d_S = nullptr, *d_Dm = nullptr, *d_B1 = nullptr, *d_B2 = nullptr, *d_C = nullptr;
  double2 *d_Kp = nullptr, *d_Ht = nullptr;  // combined-field scratch (cfg.bm_eta > 0)
  int* d_Cpiv = nullptr;
  const double2* Rroot = nullptr;
  double* d_D1 = nullptr;  // Chebyshev-Lobatto differentiation matrix (device copy)
  // mixed precision: FP32 factors (kept leaf scratch: LU(Aii), X, Ni, Kinv), FP64 refinement
  LeafScratchT<float> ws32{};
  float2 *d_R32 = nullptr, *d_Y32 = nullptr;
  std::vector<LevelOps<float2>> ops32;
  float2 *d_B2_32 = nullptr, *d_C32 = nullptr;
  int* d_Cpiv32 = nullptr;
  const float2* Rroot32 = nullptr;
  int refine_iters = 0;
  double refine_update = 0.0;
  double refine_est = 0.0;
  double bie_k = -1.0;  // wavenumber the layer-potential matrices were assembled for
  int *d_root_of_bie = nullptr, *d_bie_of_root = nullptr;  // root box order <-> boundary-node order
  double2* d_Rb = nullptr;  // root ItI map in boundary-node order (FP64)
  float2* d_Rb32 = nullptr; // same, FP32; after the build it holds C^{-1} (FP32)
  GraphSlot fgraph;     // mixed: captured factorisation (see factor_mixed)
  GraphSlot pgraph[2];  // mixed: captured refinement-pass bodies (first pass, corrections)
  double2* d_DS = nullptr;   // mixed: [D - I/2, -S] (N_b x 2 N_b), the exterior rows on [u; d_n u]
  float2* d_DS32 = nullptr;  // same, FP32
  // mixed: adjoint refinement -- per leaf edge node, where its interface or
  // exterior row lives (see adjoint_residual), and per merge level the offset
  // (in rows of nrhs) of its block in the interface-adjoint buffer
  int4* d_adj_desc = nullptr;
  // mixed: slices of the exterior rows [D - I/2, -S] (real and imaginary parts)
  // for the emulated FP64 residual product, made once per k
  char* d_ds_oz = nullptr;
  double ds_oz_k = -1.0;
  char* d_dst_oz = nullptr;  // the same rows transposed, for the adjoint refinement
  double dst_oz_k = -1.0;
  std::vector<long long> if_off;
  long long if_rows = 0;
  int adj_iters = 0;
  double adj_update = -1.0, adj_est = -1.0;
  // per-call workspace
  char* ws_base = nullptr;
  size_t ws_cap = 0;
  // the wavenumber of the current build on the device: the kernels of the
  // captured factorisation and refinement passes read it there, so one graph
  // serves every k of a sweep on this tree
  double* d_k = nullptr;
  double k_dev = 0.0;
  long long builds = 0;
  // phase times of the last build recorded launch by launch (-1 after a graph replay)
  cudaEvent_t ph_ev[3] = {nullptr, nullptr, nullptr};
  double t_interior = -1.0, t_bdry = -1.0;
};

namespace {

struct LaunchScope {
  long long* prev;
  explicit LaunchScope(hs_ctx* c) : prev(g_launch_counter) { g_launch_counter = &c->launches; }
  ~LaunchScope() { g_launch_counter = prev; }
};

int fail(hs_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

// Enqueue a fixed launch sequence on s: eagerly when `capture` is false,
// otherwise by replaying the graph in `slot`, capturing it first (stream
// capture of the same sequence) when the slot is empty or was captured for
// other (base, M, P, k).  Kernels of a replay are added to the launch count.
template <typename F>
int run_captured(hs_ctx* ctx, cudaStream_t s, GraphSlot& slot, bool capture, const void* base, int M, int P,
                 double k, F&& enqueue) {
  if (!capture) return enqueue();
  if (!slot.exec || slot.base != base || slot.M != M || slot.P != P || slot.k != k) {
    slot.reset();
    if (slot.seen_base != base || slot.seen_M != M || slot.seen_P != P || slot.seen_k != k) {
      slot.seen_base = base;
      slot.seen_M = M;
      slot.seen_P = P;
      slot.seen_k = k;
      return enqueue();
    }
    long long* counter = g_launch_counter;
    const long long before = counter ? *counter : 0;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail(ctx, HS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    const int rc = enqueue();
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    const long long kernels = counter ? *counter - before : 0;
    if (counter) *counter = before;  // counted at each replay instead
    if (rc != HS_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return rc != HS_OK ? rc : fail(ctx, HS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&slot.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      slot.exec = nullptr;
      return fail(ctx, HS_ECUDA, std::string("graph instantiation: ") + cudaGetErrorString(e));
    }
    slot.base = base;
    slot.M = M;
    slot.P = P;
    slot.k = k;
    slot.kernels = kernels;
  }
  const cudaError_t e = cudaGraphLaunch(slot.exec, s);
  if (e != cudaSuccess) return fail(ctx, HS_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  if (g_launch_counter) *g_launch_counter += slot.kernels;
  return HS_OK;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(ctx, e_ == cudaErrorMemoryAllocation ? HS_ENOMEM : HS_ECUDA, \
                                       std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

#define CKR(expr)                 \
  do {                            \
    int r_ = (expr);              \
    if (r_ != HS_OK) return r_;   \
  } while (0)

// True (and one fewer left) while the test hook says the next allocation fails.
bool injected_alloc_failure() {
  if (g_fail_allocs <= 0) return false;
  --g_fail_allocs;
  return true;
}

template <typename T> int dalloc(hs_ctx* ctx, T** p, size_t n) {
  if (injected_alloc_failure()) return fail(ctx, HS_ENOMEM, "device allocation refused (injected failure)");
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess)
    return fail(ctx, HS_ENOMEM, std::string("cudaMalloc of ") + std::to_string(n * sizeof(T)) + " bytes: " +
                                    cudaGetErrorString(e));
  ctx->allocs.push_back(v);
  *p = reinterpret_cast<T*>(v);
  return HS_OK;
}

int ensure_ws(hs_ctx* ctx, size_t bytes, Arena& a) {
  bytes += (1u << 20);  // slack for alignment padding
  if (bytes > ctx->ws_cap) {
    if (injected_alloc_failure()) return fail(ctx, HS_ENOMEM, "workspace allocation refused (injected failure)");
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->ws_base) cudaFree(ctx->ws_base);
    ctx->ws_base = nullptr;
    ctx->ws_cap = 0;
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, bytes);
    if (e != cudaSuccess) return fail(ctx, HS_ENOMEM, std::string("workspace cudaMalloc: ") + cudaGetErrorString(e));
    ctx->ws_base = (char*)v;
    ctx->ws_cap = bytes;
  }
  a.base = ctx->ws_base;
  a.cap = ctx->ws_cap;
  a.off = 0;
  return HS_OK;
}

int check_info(hs_ctx* ctx) {
  std::vector<int> info(ctx->ninfo);
  CK(cudaMemcpyAsync(info.data(), ctx->d_info, sizeof(int) * ctx->ninfo, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int v : info)
    if (v != 0) return fail(ctx, HS_ESINGULAR, "zero pivot in a factorisation (column " + std::to_string(v) + ")");
  if (tc_timed_out(ctx->stream)) return fail(ctx, HS_ETIMEOUT, "a tensor-core GEMM wait gave up");
  return HS_OK;
}

// Events bracketing the interior factorisation (leaves and merges) and the
// exterior one (layer potentials when k is new, coupling, root LU) of a build.
int phase_events(hs_ctx* ctx) {
  for (auto& e : ctx->ph_ev)
    if (!e) CK(cudaEventCreate(&e));
  return HS_OK;
}

// After the build's stream was synchronised: the two phase times in ms.
void phase_times(hs_ctx* ctx, bool recorded) {
  ctx->t_interior = ctx->t_bdry = -1.0;
  if (!recorded) return;
  float a = 0.f, b = 0.f;
  if (cudaEventElapsedTime(&a, ctx->ph_ev[0], ctx->ph_ev[1]) == cudaSuccess &&
      cudaEventElapsedTime(&b, ctx->ph_ev[1], ctx->ph_ev[2]) == cudaSuccess) {
    ctx->t_interior = a;
    ctx->t_bdry = b;
  }
}

// Tree bookkeeping: merge levels from leaves (1 x 1) to the root (nL x nL).
//
// Every leaf-edge node has a physical id: vertical edge lines x = i (i = 0..nL)
// at leaf row iy, or horizontal lines y = j at leaf column ix, node t = 1..14.
// A box's boundary is an ordered list of ids; a leaf lists S, E, N, W (each by
// increasing coordinate), and a parent lists its alpha child's exterior nodes
// then its beta child's, so every side stays in increasing coordinate order.
// The maps of one level are computed on the first pair of boxes and hold for
// every pair by translation.
struct TreeIds {
  int nL;
  int v(int i, int iy, int t) const { return (i * nL + iy) * 14 + t - 1; }
  int h(int j, int ix, int t) const { return (nL + 1) * nL * 14 + (j * nL + ix) * 14 + t - 1; }
  std::vector<int> leaf(int ix, int iy) const {
    std::vector<int> l;
    for (int t = 1; t <= 14; ++t) l.push_back(h(iy, ix, t));      // S
    for (int t = 1; t <= 14; ++t) l.push_back(v(ix + 1, iy, t));  // E
    for (int t = 1; t <= 14; ++t) l.push_back(h(iy + 1, ix, t));  // N
    for (int t = 1; t <= 14; ++t) l.push_back(v(ix, iy, t));      // W
    return l;
  }
};

struct MergeMap {
  std::vector<int> parent, I3a, I3b, src;
  int n1 = 0;
};

MergeMap merge_lists(const std::vector<int>& a, const std::vector<int>& b) {
  MergeMap m;
  std::vector<int> pos_b_sorted(b.size());
  auto find = [](const std::vector<int>& l, int id) {
    for (size_t i = 0; i < l.size(); ++i)
      if (l[i] == id) return (int)i;
    return -1;
  };
  std::vector<char> b_shared(b.size(), 0);
  std::vector<int> ext_a;
  for (size_t i = 0; i < a.size(); ++i) {
    int j = find(b, a[i]);
    if (j >= 0) {
      m.I3a.push_back((int)i);
      m.I3b.push_back(j);
      b_shared[j] = 1;
    } else {
      ext_a.push_back((int)i);
    }
  }
  for (int i : ext_a) {
    m.parent.push_back(a[i]);
    m.src.push_back(i);
  }
  m.n1 = (int)ext_a.size();
  for (size_t j = 0; j < b.size(); ++j)
    if (!b_shared[j]) {
      m.parent.push_back(b[j]);
      m.src.push_back((1 << 20) | (int)j);
    }
  return m;
}

// Boundary id list of box (px, py) at box level bl (0 = leaves; odd levels
// come from horizontal merges, even levels >= 2 from vertical ones).
std::vector<int> box_list(const TreeIds& g, int bl, int px, int py) {
  if (bl == 0) return g.leaf(px, py);
  const bool horiz = (bl % 2) == 1;
  std::vector<int> a = horiz ? box_list(g, bl - 1, 2 * px, py) : box_list(g, bl - 1, px, 2 * py);
  std::vector<int> b = horiz ? box_list(g, bl - 1, 2 * px + 1, py) : box_list(g, bl - 1, px, 2 * py + 1);
  return merge_lists(a, b).parent;
}

int setup_tree(hs_ctx* ctx) {
  const int nL = ctx->nL;
  TreeIds g{nL};
  int sx = 1, sy = 1, bl = 0;
  bool horiz = true;
  while (sx < nL || sy < nL) {
    Level L{};
    L.horiz = horiz;
    L.sx = sx;
    L.sy = sy;
    std::vector<int> la = box_list(g, bl, 0, 0);
    std::vector<int> lb = horiz ? box_list(g, bl, 1, 0) : box_list(g, bl, 0, 1);
    MergeMap mm = merge_lists(la, lb);
    const int psx = horiz ? 2 * sx : sx, psy = horiz ? sy : 2 * sy;
    L.nc = (int)la.size();
    L.ni = (int)mm.I3a.size();
    L.np = (int)mm.src.size();
    L.n1 = mm.n1;
    const int nbx_c = nL / sx, nbx_p = nL / psx, nby_p = nL / psy;
    L.nbox = nbx_p * nby_p;
    std::vector<int> al(L.nbox), be(L.nbox);
    for (int py = 0; py < nby_p; ++py)
      for (int px = 0; px < nbx_p; ++px) {
        int b = py * nbx_p + px;
        if (horiz) {
          al[b] = py * nbx_c + 2 * px;
          be[b] = al[b] + 1;
        } else {
          al[b] = (2 * py) * nbx_c + px;
          be[b] = (2 * py + 1) * nbx_c + px;
        }
      }
    CKR(dalloc(ctx, &L.d_alpha, L.nbox));
    CKR(dalloc(ctx, &L.d_beta, L.nbox));
    CKR(dalloc(ctx, &L.d_src, L.np));
    CKR(dalloc(ctx, &L.d_I3a, L.ni));
    CKR(dalloc(ctx, &L.d_I3b, L.ni));
    CK(cudaMemcpy(L.d_alpha, al.data(), sizeof(int) * L.nbox, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.d_beta, be.data(), sizeof(int) * L.nbox, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.d_src, mm.src.data(), sizeof(int) * L.np, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.d_I3a, mm.I3a.data(), sizeof(int) * L.ni, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.d_I3b, mm.I3b.data(), sizeof(int) * L.ni, cudaMemcpyHostToDevice));
    const size_t nb = L.nbox;
    L.nbx_p = nbx_p;
    if (ctx->cfg.precision == HS_FP64) {
      CKR(dalloc(ctx, &L.XZ, nb * 2 * L.ni * L.np));
      CKR(dalloc(ctx, &L.U2, nb * L.ni * L.np));
      CKR(dalloc(ctx, &L.A33, nb * L.ni * L.ni));
      CKR(dalloc(ctx, &L.B33, nb * L.ni * L.ni));
      CKR(dalloc(ctx, &L.M, nb * L.ni * L.ni));
      CKR(dalloc(ctx, &L.Mpiv, nb * L.ni));
      CKR(dalloc(ctx, &L.R, nb * (size_t)L.np * L.np));
    } else {
      LevelOps<float2> O{};
      CKR(dalloc(ctx, &O.XZ, nb * 2 * L.ni * L.np));
      CKR(dalloc(ctx, &O.U2, nb * L.ni * L.np));
      CKR(dalloc(ctx, &O.A33, nb * L.ni * L.ni));
      CKR(dalloc(ctx, &O.B33, nb * L.ni * L.ni));
      CKR(dalloc(ctx, &O.M, nb * L.ni * L.ni));
      CKR(dalloc(ctx, &O.Mpiv, nb * L.ni));
      CKR(dalloc(ctx, &O.R, nb * (size_t)L.np * L.np));
      ctx->ops32.push_back(O);
    }
    ctx->levels.push_back(L);
    sx = psx;
    sy = psy;
    horiz = !horiz;
    ++bl;
  }
  // Interface-adjoint offsets and, for the mixed path's adjoint refinement,
  // the row each leaf edge node's u and d_n u enter: the interface row of a
  // merge level (alpha or beta side) or the exterior row of a boundary node.
  // Same node arithmetic as the interface and boundary residual kernels.
  ctx->if_off.clear();
  ctx->if_rows = 0;
  for (auto& L : ctx->levels) {
    ctx->if_off.push_back(ctx->if_rows);
    ctx->if_rows += (long long)L.nbox * 2 * L.ni;
  }
  if (ctx->cfg.precision == HS_MIXED) {
    std::vector<int4> desc((size_t)nL * nL * 56, make_int4(-1, 0, -1, 0));
    for (size_t li = 0; li < ctx->levels.size(); ++li) {
      const Level& L = ctx->levels[li];
      for (int b = 0; b < L.nbox; ++b) {
        const int px = b % L.nbx_p, py = b / L.nbx_p;
        for (int t = 0; t < L.ni; ++t) {
          int la, lb, ea, eb;
          const int node = t % 14 + 1;
          if (L.horiz) {
            const int x0 = px * 2 * L.sx, y0 = py * L.sy, ly = y0 + t / 14;
            la = ly * nL + (x0 + L.sx - 1);
            lb = ly * nL + (x0 + L.sx);
            ea = 14 + node - 1;  // alpha: east edge
            eb = 42 + node - 1;  // beta: west edge
          } else {
            const int x0 = px * L.sx, y0 = py * 2 * L.sy, lx = x0 + t / 14;
            la = (y0 + L.sy - 1) * nL + lx;
            lb = (y0 + L.sy) * nL + lx;
            ea = 28 + node - 1;  // alpha: north edge
            eb = node - 1;       // beta: south edge
          }
          const int row = (int)(ctx->if_off[li] + (long long)b * 2 * L.ni + t);
          desc[(size_t)la * 56 + ea] = make_int4(row, L.ni, 0, 0);
          desc[(size_t)lb * 56 + eb] = make_int4(row, L.ni, 1, 0);
        }
      }
    }
    const int nbd = 56 * nL;
    for (int jn = 0; jn < nbd; ++jn) {
      const int side = jn / (14 * nL), i = (jn % (14 * nL)) / 14, t = jn % 14 + 1;
      int leaf, e;
      switch (side) {
        case 0: leaf = i; e = t - 1; break;
        case 1: leaf = i * nL + (nL - 1); e = 14 + t - 1; break;
        case 2: leaf = (nL - 1) * nL + i; e = 28 + t - 1; break;
        default: leaf = i * nL; e = 42 + t - 1; break;
      }
      desc[(size_t)leaf * 56 + e] = make_int4(jn, 0, 2, 0);
    }
    for (const int4& d : desc)
      if (d.z < 0) return fail(ctx, HS_EINVAL, "internal: a leaf edge node belongs to no row");
    CKR(dalloc(ctx, &ctx->d_adj_desc, desc.size()));
    CK(cudaMemcpy(ctx->d_adj_desc, desc.data(), sizeof(int4) * desc.size(), cudaMemcpyHostToDevice));
  }
  // Root order vs the order of the boundary nodes of the exterior equations
  // (S, E, N, W sides, each by increasing coordinate): root_of_bie[j] is the
  // root position of boundary node j, bie_of_root its inverse.
  std::vector<int> root = box_list(g, bl, 0, 0);
  std::vector<int> bie;
  for (int i = 0; i < nL; ++i)
    for (int t = 1; t <= 14; ++t) bie.push_back(g.h(0, i, t));
  for (int i = 0; i < nL; ++i)
    for (int t = 1; t <= 14; ++t) bie.push_back(g.v(nL, i, t));
  for (int i = 0; i < nL; ++i)
    for (int t = 1; t <= 14; ++t) bie.push_back(g.h(nL, i, t));
  for (int i = 0; i < nL; ++i)
    for (int t = 1; t <= 14; ++t) bie.push_back(g.v(0, i, t));
  const int nb = (int)bie.size();
  if ((int)root.size() != nb) return fail(ctx, HS_EINVAL, "internal: root boundary size mismatch");
  std::vector<int> root_of_bie(nb, -1), bie_of_root(nb, -1);
  for (int j = 0; j < nb; ++j) {
    for (int r = 0; r < nb; ++r)
      if (root[r] == bie[j]) {
        root_of_bie[j] = r;
        bie_of_root[r] = j;
        break;
      }
    if (root_of_bie[j] < 0) return fail(ctx, HS_EINVAL, "internal: boundary node missing from the root");
  }
  CKR(dalloc(ctx, &ctx->d_root_of_bie, nb));
  CKR(dalloc(ctx, &ctx->d_bie_of_root, nb));
  CK(cudaMemcpy(ctx->d_root_of_bie, root_of_bie.data(), sizeof(int) * nb, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_bie_of_root, bie_of_root.data(), sizeof(int) * nb, cudaMemcpyHostToDevice));
  return HS_OK;
}

int setup_boundary(hs_ctx* ctx) {
  const int nL = ctx->nL;
  const double h = ctx->h;
  std::vector<double> t = lobatto(16);
  std::vector<double> tin(t.begin() + 1, t.end() - 1);
  std::vector<double> wf = fejer2(14);
  const int npanel = 4 * nL, nb = npanel * 14;
  std::vector<double> x(nb), y(nb), nx(nb), ny(nb), w(nb);
  std::vector<int> panel(nb);
  std::vector<double> p0x(npanel), p0y(npanel), tx(npanel), ty(npanel), pnx(npanel), pny(npanel);
  for (int side = 0; side < 4; ++side)
    for (int i = 0; i < nL; ++i) {
      int q = side * nL + i;
      double sx0, sy0, tX, tY, nX, nY;
      switch (side) {
        case 0: sx0 = -1.0 + i * h; sy0 = -1.0; tX = 1; tY = 0; nX = 0; nY = -1; break;  // S
        case 1: sx0 = 1.0; sy0 = -1.0 + i * h; tX = 0; tY = 1; nX = 1; nY = 0; break;    // E
        case 2: sx0 = -1.0 + i * h; sy0 = 1.0; tX = 1; tY = 0; nX = 0; nY = 1; break;    // N
        default: sx0 = -1.0; sy0 = -1.0 + i * h; tX = 0; tY = 1; nX = -1; nY = 0; break; // W
      }
      p0x[q] = sx0; p0y[q] = sy0; tx[q] = tX; ty[q] = tY; pnx[q] = nX; pny[q] = nY;
      for (int a = 0; a < 14; ++a) {
        int j = q * 14 + a;
        double s = (tin[a] + 1.0) * h / 2.0;
        x[j] = sx0 + s * tX;
        y[j] = sy0 + s * tY;
        nx[j] = nX;
        ny[j] = nY;
        w[j] = wf[a] * h / 2.0;
        panel[j] = q;
      }
    }
  // near panels: segment distance <= h (the panel itself, two on each side
  // along the boundary, wrapping around the corners)
  std::vector<int> nearp(npanel * 5, -1);
  auto segdist = [&](int p, int q) {
    auto ptseg = [&](double px, double py, int s) {
      double dx = tx[s] * h, dy = ty[s] * h;
      double u = ((px - p0x[s]) * dx + (py - p0y[s]) * dy) / (dx * dx + dy * dy);
      u = std::min(1.0, std::max(0.0, u));
      double ex = px - (p0x[s] + u * dx), ey = py - (p0y[s] + u * dy);
      return std::sqrt(ex * ex + ey * ey);
    };
    double e1x = p0x[p] + tx[p] * h, e1y = p0y[p] + ty[p] * h;
    double e2x = p0x[q] + tx[q] * h, e2y = p0y[q] + ty[q] * h;
    return std::min(std::min(ptseg(p0x[p], p0y[p], q), ptseg(e1x, e1y, q)),
                    std::min(ptseg(p0x[q], p0y[q], p), ptseg(e2x, e2y, p)));
  };
  for (int p = 0; p < npanel; ++p) {
    int c = 0;
    for (int q = 0; q < npanel && c < 5; ++q)
      if (segdist(p, q) <= h * (1 + 1e-9)) nearp[p * 5 + c++] = q;
  }
  Boundary& B = ctx->B;
  B.nb = nb;
  B.npanel = npanel;
  B.h = h;
  CKR(dalloc(ctx, &B.x, nb)); CKR(dalloc(ctx, &B.y, nb)); CKR(dalloc(ctx, &B.nx, nb)); CKR(dalloc(ctx, &B.ny, nb));
  CKR(dalloc(ctx, &B.w, nb)); CKR(dalloc(ctx, &B.panel, nb));
  CKR(dalloc(ctx, &B.p0x, npanel)); CKR(dalloc(ctx, &B.p0y, npanel)); CKR(dalloc(ctx, &B.tx, npanel));
  CKR(dalloc(ctx, &B.ty, npanel)); CKR(dalloc(ctx, &B.pnx, npanel)); CKR(dalloc(ctx, &B.pny, npanel));
  CKR(dalloc(ctx, &B.near, npanel * 5));
  CK(cudaMemcpy(B.x, x.data(), sizeof(double) * nb, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(B.y, y.data(), sizeof(double) * nb, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(B.nx, nx.data(), sizeof(double) * nb, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(B.ny, ny.data(), sizeof(double) * nb, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(B.w, w.data(), sizeof(double) * nb, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(B.panel, panel.data(), sizeof(int) * nb, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(B.p0x, p0x.data(), sizeof(double) * npanel, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(B.p0y, p0y.data(), sizeof(double) * npanel, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(B.tx, tx.data(), sizeof(double) * npanel, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(B.ty, ty.data(), sizeof(double) * npanel, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(B.pnx, pnx.data(), sizeof(double) * npanel, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(B.pny, pny.data(), sizeof(double) * npanel, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(B.near, nearp.data(), sizeof(int) * npanel * 5, cudaMemcpyHostToDevice));
  // quadrature constants
  std::vector<double> glx, glw;
  gauss_legendre(16, glx, glw);
  std::vector<double> lagden(14);
  for (int j = 0; j < 14; ++j) {
    double p = 1.0;
    for (int l = 0; l < 14; ++l)
      if (l != j) p *= (tin[j] - tin[l]);
    lagden[j] = p;
  }
  std::vector<double> dref = diff_matrix(tin);  // panel-node differentiation, [l][j] = L_j'(t_l)
  upload_quad_constants(glx.data(), glw.data(), tin.data(), lagden.data(), dref.data(), ctx->stream);
  std::vector<double> D1 = diff_matrix(t);
  upload_cheb_diff(D1.data(), ctx->stream);
  // root system
  const size_t nn = (size_t)nb * nb;
  CKR(dalloc(ctx, &ctx->d_S, nn));
  CKR(dalloc(ctx, &ctx->d_Dm, nn));
  if (ctx->cfg.bm_eta > 0.0) {  // K' and the tangential derivative of S for the combined-field rows
    CKR(dalloc(ctx, &ctx->d_Kp, nn));
    CKR(dalloc(ctx, &ctx->d_Ht, nn));
  }
  CKR(dalloc(ctx, &ctx->d_B1, nn));
  CKR(dalloc(ctx, &ctx->d_B2, nn));
  if (ctx->cfg.precision == HS_FP64) {
    CKR(dalloc(ctx, &ctx->d_C, nn));
    CKR(dalloc(ctx, &ctx->d_Cpiv, nb));
    CKR(dalloc(ctx, &ctx->d_Rb, nn));
  } else {
    CKR(dalloc(ctx, &ctx->d_Rb32, nn));
    CKR(dalloc(ctx, &ctx->d_B2_32, nn));
    CKR(dalloc(ctx, &ctx->d_C32, nn));
    CKR(dalloc(ctx, &ctx->d_Cpiv32, nb));
    CKR(dalloc(ctx, &ctx->d_DS, 2 * nn));
    CKR(dalloc(ctx, &ctx->d_DS32, 2 * nn));
  }
  CKR(dalloc(ctx, &ctx->d_D1, 256));
  CK(cudaMemcpy(ctx->d_D1, D1.data(), sizeof(double) * 256, cudaMemcpyHostToDevice));
  return HS_OK;
}

int setup(hs_ctx* ctx) {
  const int nL = ctx->nL;
  ctx->nleaf = nL * nL;
  ctx->n14 = 14 * nL;
  ctx->n16 = 16 * nL;
  ctx->h = 2.0 / nL;
  ctx->chunk = std::min(ctx->nleaf, 1024);
  std::vector<double> t = lobatto(16);
  std::vector<double> xg(ctx->n16), xint(ctx->n14);
  for (int ix = 0; ix < nL; ++ix)
    for (int a = 0; a < 16; ++a) {
      double xv = -1.0 + ix * ctx->h + (t[a] + 1.0) * ctx->h / 2.0;
      xg[ix * 16 + a] = xv;
      if (a >= 1 && a <= 14) xint[ix * 14 + a - 1] = xv;
    }
  CKR(dalloc(ctx, &ctx->d_xg, ctx->n16));
  CKR(dalloc(ctx, &ctx->d_xint, ctx->n14));
  CK(cudaMemcpy(ctx->d_xg, xg.data(), sizeof(double) * ctx->n16, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_xint, xint.data(), sizeof(double) * ctx->n14, cudaMemcpyHostToDevice));
  const int S1 = ctx->cfg.S1, S2 = ctx->cfg.S2;
  CKR(dalloc(ctx, &ctx->d_q, (size_t)ctx->nleaf * 256));
  CKR(dalloc(ctx, &ctx->d_c, (size_t)S1 * S2));
  CKR(dalloc(ctx, &ctx->d_sx16, (size_t)S1 * ctx->n16));
  CKR(dalloc(ctx, &ctx->d_sy16, (size_t)S2 * ctx->n16));
  CKR(dalloc(ctx, &ctx->d_T, (size_t)S1 * ctx->n16));
  CKR(dalloc(ctx, &ctx->d_Qg, (size_t)ctx->n16 * ctx->n16));
  CKR(dalloc(ctx, &ctx->d_sxi, (size_t)S1 * ctx->n14));
  CKR(dalloc(ctx, &ctx->d_syi, (size_t)S2 * ctx->n14));
  ctx->ninfo = std::max(ctx->nleaf, 16) + 1;
  CKR(dalloc(ctx, &ctx->d_info, ctx->ninfo));
  CKR(dalloc(ctx, &ctx->d_k, 1));
  // leaf factors and scratch
  const size_t nl = ctx->nleaf;
  if (ctx->cfg.precision == HS_FP64) {
    const size_t ch = ctx->chunk;
    CKR(dalloc(ctx, &ctx->d_Rleaf, nl * NE * NE));
    CKR(dalloc(ctx, &ctx->d_Y, nl * NL * NE));
    CKR(dalloc(ctx, &ctx->d_Q, nl * NI * NE));
    LeafScratch& w = ctx->ws;
    CKR(dalloc(ctx, &w.Aii, ch * NI * NI));
    CKR(dalloc(ctx, &w.Aie, ch * NI * NE));
    CKR(dalloc(ctx, &w.Ni, ch * NE * NI));
    CKR(dalloc(ctx, &w.NiT, ch * NI * NE));
    CKR(dalloc(ctx, &w.Ne, ch * NE * NE));
    CKR(dalloc(ctx, &w.K, ch * NE * NE));
    CKR(dalloc(ctx, &w.Kinv, ch * NE * NE));
    CKR(dalloc(ctx, &w.piv, ch * NI));
    CKR(dalloc(ctx, &w.pivK, ch * NE));
    if (ctx->cfg.leaf_impedance) {
      CKR(dalloc(ctx, &w.L, ch * NL * NL));
      CKR(dalloc(ctx, &w.Et, ch * NL * NE));
      CKR(dalloc(ctx, &w.pivL, ch * NL));
    }
  } else {
    // every leaf's factors are kept: the refinement's particular solves reuse them
    CKR(dalloc(ctx, &ctx->d_R32, nl * NE * NE));
    CKR(dalloc(ctx, &ctx->d_Y32, nl * NL * NE));
    LeafScratchT<float>& w = ctx->ws32;
    CKR(dalloc(ctx, &w.Aii, nl * NI * NI));
    CKR(dalloc(ctx, &w.Aie, nl * NI * NE));
    CKR(dalloc(ctx, &w.Ni, nl * NE * NI));
    CKR(dalloc(ctx, &w.NiT, nl * NI * NE));
    CKR(dalloc(ctx, &w.Ne, nl * NE * NE));
    CKR(dalloc(ctx, &w.K, nl * NE * NE));
    CKR(dalloc(ctx, &w.Kinv, nl * NE * NE));
    CKR(dalloc(ctx, &w.piv, nl * NI));
    CKR(dalloc(ctx, &w.pivK, nl * NE));
    CKR(dalloc(ctx, &w.Ainv, nl * NI * NI));
    if (ctx->cfg.leaf_impedance) {  // every leaf's impedance system and particular-solution operator
      CKR(dalloc(ctx, &w.L, nl * NL * NL));
      CKR(dalloc(ctx, &w.pivL, nl * NL));
      CKR(dalloc(ctx, &w.P, nl * NL * NI));
    }
  }
  CKR(setup_tree(ctx));
  CKR(setup_boundary(ctx));
  CK(cudaStreamSynchronize(ctx->stream));
  return HS_OK;
}

// The wavenumber of the build into the device scalar the kernels read.
int set_device_k(hs_ctx* ctx, cudaStream_t s, double k) {
  ctx->k_dev = k;
  CK(cudaMemcpyAsync(ctx->d_k, &ctx->k_dev, sizeof(double), cudaMemcpyHostToDevice, s));
  return HS_OK;
}

// The layer-potential matrices of the mixed path for a new k (S, D - I/2, B1,
// B2 and the stacked exterior rows in FP64 and FP32): they depend on k and the
// boundary only.
void assemble_exterior_mixed(hs_ctx* ctx, cudaStream_t s, double k) {
  const int nb = ctx->B.nb;
  const long long nn = (long long)nb * nb;
  bie_matrices(s, ctx->B, k, ctx->d_S, ctx->d_Dm);
  if (ctx->cfg.bm_eta > 0.0) bie_combined(s, ctx->B, k, ctx->cfg.bm_eta, ctx->d_S, ctx->d_Dm, ctx->d_Kp, ctx->d_Ht);
  bie_root_ops(s, nb, k, ctx->d_S, ctx->d_Dm, ctx->d_B1, ctx->d_B2);
  convert_d2f(s, ctx->d_B2, ctx->d_B2_32, nn);
  stack_exterior(s, ctx->d_Dm, ctx->d_S, nb, ctx->d_DS, ctx->d_DS32);
  ctx->bie_k = k;
}

// FP32 factors of the mixed-precision path: leaves, merges and the coupled
// root system in complex FP32; the layer-potential matrices stay in FP64 for
// the refinement residual.
// Device work of the mixed-precision factorisation (no host synchronisation,
// so that it can be captured into a CUDA graph).
int enqueue_factor_mixed(hs_ctx* ctx, double k, cudaStream_t s, bool record) {
  CK(cudaMemsetAsync(ctx->d_info, 0, sizeof(int) * ctx->ninfo, s));
  if (record) CK(cudaEventRecord(ctx->ph_ev[0], s));
  if (ctx->cfg.leaf_impedance)
    leaf_build_chunk_impedance<float>(s, ctx->d_q, 0, ctx->nleaf, k, ctx->d_k, ctx->h, ctx->ws32, ctx->d_R32,
                                      ctx->d_Y32, nullptr, ctx->d_info);
  else
    leaf_build_chunk<float>(s, ctx->d_q, 0, ctx->nleaf, k, ctx->d_k, ctx->h, ctx->ws32, ctx->d_R32, ctx->d_Y32,
                            nullptr, ctx->d_info);
  const float2* Rc = ctx->d_R32;
  for (size_t li = 0; li < ctx->levels.size(); ++li) {
    merge_level<float2>(s, ctx->levels[li], ctx->ops32[li], Rc, ctx->d_info);
    Rc = ctx->ops32[li].R;
  }
  if (record) CK(cudaEventRecord(ctx->ph_ev[1], s));
  const int nb = ctx->B.nb;
  permute_square<float2>(s, Rc, ctx->d_root_of_bie, nb, ctx->d_Rb32);  // root map in boundary-node order
  const long long nn = (long long)nb * nb;
  // a new k's layer potentials (the captured sequence never holds them: before a
  // replay they are assembled eagerly, see factor_mixed)
  if (ctx->bie_k != k) assemble_exterior_mixed(ctx, s, k);
  convert_d2f(s, ctx->d_B1, ctx->d_C32, nn);
  gemm<float2, float2, float2>(s, OP_N, OP_N, nb, nb, nb, make_float2(-1.f, 0.f), ctx->d_B2_32, nb, 0, ctx->d_Rb32,
                               nb, 0, make_float2(1.f, 0.f), ctx->d_C32, nb, 0, 1);
  lu_factor<float2>(s, ctx->d_C32, nb, 0, nb, ctx->d_Cpiv32, 0, ctx->d_info, 1);
  // C^{-1} explicitly (in the buffer of the root map, no longer needed): each
  // refinement pass then applies it with one GEMM
  lu_inverse<float2>(s, ctx->d_C32, nb, 0, nb, ctx->d_Cpiv32, 0, ctx->d_Rb32, nb, 0, 1);
  if (record) CK(cudaEventRecord(ctx->ph_ev[2], s));
  CK(cudaGetLastError());
  return HS_OK;
}

// Mixed-precision factorisation.  The first build of a context runs eagerly
// (its phases are timed); every later build, at any k, replays a CUDA graph of
// the same launch sequence (about 900 launches: leaf factors, every merge
// level, the root), captured at the second build: the kernels read k from
// device memory, and a new k's layer-potential matrices are assembled eagerly
// before the replay.  This removes the per-launch host overhead and the gaps
// between the many small kernels at every frequency of a sweep.
int factor_mixed(hs_ctx* ctx, double k) {
  cudaStream_t s = ctx->stream;
  Phase ph("hs_factor_mixed");
  CKR(set_device_k(ctx, s, k));
  // (per-launch profiling of the FP32 families needs eager launches; the
  // factorisation has no FP64 GEMM, so FP64 profiling does not prevent it)
  const bool graph = g_use_graphs && ctx->builds > 0 && !prof_active(2) && !prof_active(3);
  if (!graph) CKR(phase_events(ctx));
  if (graph && ctx->bie_k != k) assemble_exterior_mixed(ctx, s, k);
  CKR(run_captured(ctx, s, ctx->fgraph, graph, nullptr, 0, 0, 0.0,
                   [&] { return enqueue_factor_mixed(ctx, k, s, !graph); }));
  ctx->Rroot32 = nullptr;
  CKR(check_info(ctx));
  phase_times(ctx, !graph);
  ctx->k = k;
  ctx->built = true;
  ++ctx->builds;
  return HS_OK;
}

// Factor the operator for the q currently in d_q (Sec. 2).
int factor(hs_ctx* ctx, double k) {
  if (ctx->cfg.precision == HS_MIXED) return factor_mixed(ctx, k);
  cudaStream_t s = ctx->stream;
  CKR(phase_events(ctx));
  CKR(set_device_k(ctx, s, k));
  CK(cudaMemsetAsync(ctx->d_info, 0, sizeof(int) * ctx->ninfo, s));
  CK(cudaEventRecord(ctx->ph_ev[0], s));
  Phase ph("hs_factor_fp64");
  for (int l0 = 0; l0 < ctx->nleaf; l0 += ctx->chunk) {
    int n = std::min(ctx->chunk, ctx->nleaf - l0);
    if (ctx->cfg.leaf_impedance)
      leaf_build_chunk_impedance<double>(s, ctx->d_q, l0, n, k, ctx->d_k, ctx->h, ctx->ws,
                                 ctx->d_Rleaf + (size_t)l0 * NE * NE, ctx->d_Y + (size_t)l0 * NL * NE,
                                 ctx->d_Q + (size_t)l0 * NI * NE, ctx->d_info);
    else
      leaf_build_chunk(s, ctx->d_q, l0, n, k, ctx->d_k, ctx->h, ctx->ws, ctx->d_Rleaf + (size_t)l0 * NE * NE,
                       ctx->d_Y + (size_t)l0 * NL * NE, ctx->d_Q + (size_t)l0 * NI * NE, ctx->d_info);
  }
  const double2* Rc = ctx->d_Rleaf;
  {
    Phase pm("hs_merges");
    for (auto& L : ctx->levels) {
      merge_level(s, L, Rc, ctx->d_info);
      Rc = L.R;
    }
  }
  CK(cudaEventRecord(ctx->ph_ev[1], s));
  Phase pr("hs_root_coupling");
  const int nb = ctx->B.nb;
  permute_square<double2>(s, Rc, ctx->d_root_of_bie, nb, ctx->d_Rb);  // root map in boundary-node order
  ctx->Rroot = ctx->d_Rb;
  if (ctx->bie_k != k) {  // S, D - I/2 (or their combined-field forms), B1, B2 depend on k and the boundary only
    bie_matrices(s, ctx->B, k, ctx->d_S, ctx->d_Dm);
    if (ctx->cfg.bm_eta > 0.0) bie_combined(s, ctx->B, k, ctx->cfg.bm_eta, ctx->d_S, ctx->d_Dm, ctx->d_Kp, ctx->d_Ht);
    bie_root_ops(s, nb, k, ctx->d_S, ctx->d_Dm, ctx->d_B1, ctx->d_B2);
    ctx->bie_k = k;
  }
  // C = B1 - B2 R_root   (coupling of the interior impedances to the exterior identity)
  CK(cudaMemcpyAsync(ctx->d_C, ctx->d_B1, sizeof(double2) * nb * nb, cudaMemcpyDeviceToDevice, s));
  gemm<double2, double2, double2>(s, OP_N, OP_N, nb, nb, nb, make_double2(-1, 0), ctx->d_B2, nb, 0, ctx->Rroot, nb, 0,
                                  make_double2(1, 0), ctx->d_C, nb, 0, 1);
  lu_factor<double2>(s, ctx->d_C, nb, 0, nb, ctx->d_Cpiv, 0, ctx->d_info, 1);
  CK(cudaEventRecord(ctx->ph_ev[2], s));
  CK(cudaGetLastError());
  CKR(check_info(ctx));
  phase_times(ctx, true);
  ctx->k = k;
  ctx->built = true;
  return HS_OK;
}

// Root impedances f (nb x M) for plane waves; also returns ui, dni, g.
int root_solve(hs_ctx* ctx, cudaStream_t s, const double* alphas, int M, double2* ui, double2* dni, double2* f,
               double2* g) {
  const int nb = ctx->B.nb;
  const double2 one = make_double2(1, 0), mone = make_double2(-1, 0), zero = make_double2(0, 0);
  incident_plane(s, ctx->B, ctx->k, alphas, M, ui, dni);
  // rhs = (D - I/2) u_inc - S d_n u_inc
  gemm<double2, double2, double2>(s, OP_N, OP_N, nb, M, nb, one, ctx->d_Dm, nb, 0, ui, M, 0, zero, f, M, 0, 1);
  gemm<double2, double2, double2>(s, OP_N, OP_N, nb, M, nb, mone, ctx->d_S, nb, 0, dni, M, 0, one, f, M, 0, 1);
  lu_solve<double2>(s, OP_N, ctx->d_C, nb, 0, nb, ctx->d_Cpiv, 0, f, M, 0, M, 1);
  gemm<double2, double2, double2>(s, OP_N, OP_N, nb, M, nb, one, ctx->Rroot, nb, 0, f, M, 0, zero, g, M, 0, 1);
  return HS_OK;
}

// Downward sweep from root impedances f (nb x nrhs) to leaf fields (nleaf x 252 x nrhs).
int sweep_down(hs_ctx* ctx, cudaStream_t s, const double2* f, int nrhs, double2* bufA, double2* bufB, double2* T3,
               double2* Uleaf) {
  Phase ph("hs_sweep_down");
  permute_rows<double2>(s, f, ctx->d_bie_of_root, ctx->B.nb, nrhs, bufB);  // root box order
  const double2* Fp = bufB;
  double2* out = bufA;
  for (int li = (int)ctx->levels.size() - 1; li >= 0; --li) {
    const Level& L = ctx->levels[li];
    sweep_down_level(s, L, Fp, T3, out, nrhs);
    Fp = out;
    out = (out == bufA) ? bufB : bufA;
  }
  gemm<double2, double2, double2>(s, OP_N, OP_N, NL, nrhs, NE, make_double2(1, 0), ctx->d_Y, NE, (long long)NL * NE, Fp,
                                  nrhs, (long long)NE * nrhs, make_double2(0, 0), Uleaf, nrhs, (long long)NL * nrhs,
                                  ctx->nleaf);
  return HS_OK;
}

// Adjoint sweep for the receiver functionals: Z (nleaf x 196 x P).
int sweep_adjoint(hs_ctx* ctx, cudaStream_t s, const double2* A2, int P, double2* E, double2* CP, double2* bufA,
                  double2* bufB, double2* MU, double2* Zleaf) {
  const int nb = ctx->B.nb;
  const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
  Phase ph("hs_adjoint_sweep");
  adjoint_root_init(s, nb, P, ctx->k, A2, E, CP);
  gemm<double2, double2, double2>(s, OP_T, OP_N, nb, P, nb, one, ctx->Rroot, nb, 0, E, P, 0, one, CP, P, 0, 1);
  lu_solve<double2>(s, OP_T, ctx->d_C, nb, 0, nb, ctx->d_Cpiv, 0, CP, P, 0, P, 1);
  gemm<double2, double2, double2>(s, OP_T, OP_N, nb, P, nb, one, ctx->d_B2, nb, 0, CP, P, 0, one, E, P, 0, 1);
  permute_rows<double2>(s, E, ctx->d_bie_of_root, nb, P, bufB);  // root box order
  const double2* Lp = bufB;
  double2* out = bufA;
  for (int li = (int)ctx->levels.size() - 1; li >= 0; --li) {
    const Level& L = ctx->levels[li];
    sweep_adjoint_level(s, L, Lp, MU, out, P);
    Lp = out;
    out = (out == bufA) ? bufB : bufA;
  }
  gemm<double2, double2, double2>(s, OP_N, OP_N, NI, P, NE, one, ctx->d_Q, NE, (long long)NI * NE, Lp, P,
                                  (long long)NE * P, zero, Zleaf, P, (long long)NI * P, ctx->nleaf);
  return HS_OK;
}

size_t field_buf_elems(hs_ctx* ctx, int nrhs) {
  size_t m = (size_t)ctx->nleaf * NE;
  for (auto& L : ctx->levels) m = std::max(m, (size_t)L.nbox * 2 * L.nc);
  return m * nrhs;
}
size_t t3_elems(hs_ctx* ctx, int nrhs) {
  size_t m = 1;
  for (auto& L : ctx->levels) m = std::max(m, (size_t)L.nbox * 2 * L.ni);
  return m * nrhs;
}

int check_ctx(hs_ctx* ctx, bool need_built) {
  if (!ctx) return HS_EINVAL;
  if (need_built && !ctx->built) return fail(ctx, HS_ENOTBUILT, "hs_build has not been called");
  cudaError_t e = cudaSetDevice(ctx->cfg.device);
  if (e != cudaSuccess) return fail(ctx, HS_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  return HS_OK;
}

cudaStream_t pick(hs_ctx* ctx, void* stream) { return stream ? (cudaStream_t)stream : ctx->stream; }

// Real and imaginary parts of a complex matrix (rows x k, leading dimension
// ld, interleaved) as strided real views for slicing.
OzView re_view(const double2* A, int ld, int part) {
  return OzView{const_cast<double*>(reinterpret_cast<const double*>(A)) + part, 0, 2LL * ld, 0, 2, 1};
}
// The same for the transpose of a k x rows complex matrix (row index along its columns).
OzView re_view_t(const double2* A, int ld, int part) {
  return OzView{const_cast<double*>(reinterpret_cast<const double*>(A)) + part, 0, 2, 0, 2LL * ld, 1};
}

// Far field for M incidences into ufar (device, M x P complex).
int mixed_solve(hs_ctx* ctx, cudaStream_t s, const double* alphas, int M, const double* thetas, int P, double2* ufar,
                double2* Xout, Arena& a);
size_t mixed_bytes(hs_ctx* ctx, int M, int P);

int solve_into(hs_ctx* ctx, cudaStream_t s, const double* alphas, int M, const double* thetas, int P, double2* ufar) {
  const int nb = ctx->B.nb;
  Arena a;
  if (ctx->cfg.precision == HS_MIXED) {
    CKR(ensure_ws(ctx, mixed_bytes(ctx, M, P), a));
    return mixed_solve(ctx, s, alphas, M, thetas, P, ufar, nullptr, a);
  }
  size_t need = 4 * Arena::bytes((size_t)nb * M, 16) + Arena::bytes((size_t)2 * nb * M, 16) +
                Arena::bytes((size_t)P * 2 * nb, 16);
  CKR(ensure_ws(ctx, need, a));
  double2 *ui = a.get<double2>((size_t)nb * M), *dni = a.get<double2>((size_t)nb * M);
  double2 *f = a.get<double2>((size_t)nb * M), *g = a.get<double2>((size_t)nb * M);
  double2* PS = a.get<double2>((size_t)2 * nb * M);
  double2* A2 = a.get<double2>((size_t)P * 2 * nb);
  if (a.over) return fail(ctx, HS_ENOMEM, "workspace request beyond its sizing");
  CKR(root_solve(ctx, s, alphas, M, ui, dni, f, g));
  boundary_data(s, nb, M, ctx->k, f, g, ui, dni, PS);
  farfield_matrix(s, ctx->B, ctx->k, ctx->cfg.R, thetas, P, A2);
  gemm<double2, double2, double2>(s, OP_T, OP_T, M, P, 2 * nb, make_double2(1, 0), PS, M, 0, A2, 2 * nb, 0,
                                  make_double2(0, 0), ufar, P, 0, 1);
  CK(cudaGetLastError());
  return HS_OK;
}

size_t s3_elems(hs_ctx* ctx, int nrhs) {
  size_t m = 1;
  for (auto& L : ctx->levels) m = std::max(m, (size_t)L.nbox * 2 * L.ni);
  return m * nrhs;
}

size_t mixed_bytes(hs_ctx* ctx, int M, int P) {
  const size_t nb = ctx->B.nb, nl = ctx->nleaf;
  size_t b = 6 * Arena::bytes(nb * M, 16) + Arena::bytes(2 * nb * M, 16) + Arena::bytes((size_t)P * 2 * nb, 16) +
             Arena::bytes((size_t)M * P, 16) + Arena::bytes(2 * nb * M, 8) + Arena::bytes((size_t)P * 2 * nb, 8) +
             Arena::bytes((size_t)M * P, 8) + Arena::bytes(8, 8) + Arena::bytes(nl * NL * M, 16);
  b += Arena::bytes(nl * NL * M, 8) + 2 * Arena::bytes(field_buf_elems(ctx, M), 8) + Arena::bytes(nl * NE * M, 8) +
       Arena::bytes(nl * NI * M, 8) +
       Arena::bytes(s3_elems(ctx, M), 8) + 2 * Arena::bytes(nb * M, 8);
  for (auto& L : ctx->levels) b += Arena::bytes((size_t)L.nbox * 2 * L.ni * M, 8);
  if (g_oz_enabled)
    b += 2 * std::max(oz_wide_bytes(M, 2 * (int)nb, false),
                      oz_wide_bytes(M, 2 * (int)nb, true) + oz_wide_bytes(P, 2 * (int)nb, false)) +
         4 * std::max(oz_partial_bytes((int)nb, M, 2 * (int)nb), oz_partial_bytes(M, P, 2 * (int)nb));
  return b;
}

// Mixed-precision forward solve: FP32 direct solves as the inner solver of
// FP64 iterative refinement on the residual of the whole discrete system
// (leaf PDE rows, interface continuity rows, exterior rows).  The first pass
// is the plain FP32 solve; every later pass solves for the correction with
// body loads (the PDE residual), interface right-hand sides (continuity
// residual) and the exterior residual.  Stops when the estimated relative
// error of the far field is below tol (default 1e-9): the relative change of
// the last pass, scaled by rho / (1 - rho) once two changes give the
// contraction rate rho of the passes (rho ~ 1e-4 here, so three passes
// usually suffice); fails with HS_ENOCONV after max_iter passes.
// ufar (M x P) and/or X (FP64 leaf fields, [leaf][252][M]) may be NULL.
int mixed_solve(hs_ctx* ctx, cudaStream_t s, const double* alphas, int M, const double* thetas, int P, double2* ufar,
                double2* Xout, Arena& a) {
  const int nb = ctx->B.nb, nl = ctx->nleaf, nlev = (int)ctx->levels.size();
  const size_t nbM = (size_t)nb * M, nX = (size_t)nl * NL * M;
  const double eta = ctx->k;
  const double tol = ctx->cfg.refine_tol > 0 ? ctx->cfg.refine_tol : 1e-9;
  const int max_iter = ctx->cfg.refine_max_iter > 0 ? ctx->cfg.refine_max_iter : 8;
  const double2 one = make_double2(1, 0), mone = make_double2(-1, 0), zero = make_double2(0, 0);
  const float2 fone = make_float2(1.f, 0.f), fzero = make_float2(0.f, 0.f);
  double2 *ui = a.get<double2>(nbM), *dni = a.get<double2>(nbM);
  double2 *ub = a.get<double2>(nbM), *psib = a.get<double2>(nbM), *rext = a.get<double2>(nbM);
  double2* PS = a.get<double2>(2 * nbM);
  double2* A2 = a.get<double2>((size_t)P * 2 * nb);
  double2* uf = a.get<double2>((size_t)M * P);
  float2* PS32 = a.get<float2>(2 * nbM);
  float2* A2_32 = a.get<float2>((size_t)P * 2 * nb);
  float2* duf = a.get<float2>((size_t)M * P);
  double* nrm = a.get<double>(8);
  double2* X = a.get<double2>(nX);
  float2* Up = a.get<float2>(nX);
  float2 *B0 = a.get<float2>(field_buf_elems(ctx, M)), *B1 = a.get<float2>(field_buf_elems(ctx, M));
  float2* tmp = a.get<float2>((size_t)nl * NE * M);
  float2* wtmp = a.get<float2>((size_t)nl * NI * M);
  float2* S3 = a.get<float2>(s3_elems(ctx, M));
  float2 *f32 = a.get<float2>(nbM), *r32 = a.get<float2>(nbM);
  std::vector<float2*> TT(nlev);
  for (int li = 0; li < nlev; ++li) TT[li] = a.get<float2>((size_t)ctx->levels[li].nbox * 2 * ctx->levels[li].ni * M);
  // emulated FP64 products: slices of the boundary data (as the right operand of
  // the exterior residual, then as the left operand of the far field) and of
  // the receiver matrix
  const bool emu = g_oz_enabled;
  const size_t ob_ps = emu ? oz_wide_bytes(M, 2 * nb, false) : 0;
  const size_t ob_psa = emu ? oz_wide_bytes(M, 2 * nb, true) : 0, ob_a2 = emu ? oz_wide_bytes(P, 2 * nb, false) : 0;
  const size_t ob_part = emu ? std::max(oz_partial_bytes(nb, M, 2 * nb), oz_partial_bytes(M, P, 2 * nb)) : 0;
  char* ozs = emu ? a.get<char>(2 * std::max(ob_ps, ob_psa + ob_a2)) : nullptr;
  char* ozp = emu ? a.get<char>(4 * ob_part) : nullptr;
  if (a.over) return fail(ctx, HS_ENOMEM, "workspace request beyond its sizing");
  const size_t ob_ds = oz_wide_bytes(nb, 2 * nb, true);
  if (emu && ctx->ds_oz_k != ctx->bie_k) {  // the exterior rows of this k, sliced once
    if (!ctx->d_ds_oz) CKR(dalloc(ctx, &ctx->d_ds_oz, 2 * ob_ds));
    oz_slice_wide(s, re_view(ctx->d_DS, 2 * nb, 0), nb, 2 * nb, true, ctx->d_ds_oz);
    oz_slice_wide(s, re_view(ctx->d_DS, 2 * nb, 1), nb, 2 * nb, true, ctx->d_ds_oz + ob_ds);
    ctx->ds_oz_k = ctx->bie_k;
  }

  incident_plane(s, ctx->B, ctx->k, alphas, M, ui, dni);
  farfield_matrix(s, ctx->B, ctx->k, ctx->cfg.R, thetas, P, A2);
  convert_d2f(s, A2, A2_32, (long long)P * 2 * nb);
  CK(cudaMemsetAsync(X, 0, sizeof(double2) * nX, s));
  ctx->refine_iters = 0;
  ctx->refine_update = -1.0;
  ctx->refine_est = -1.0;
  double prev_upd = 0.0, uf0_n2 = 0.0;
  bool converged = false;
  for (int it = 0; it < max_iter; ++it) {
    Phase pp("hs_refine_pass");
    if (it > 0) {
      // FP64 residual of every row for the current iterate X; the exterior
      // rows: (D - I/2)(u_inc - u) - S (d_n u_inc - d_n u) = -[D - I/2, -S] [u_s; d_n u_s]
      residual_pde(s, X, ctx->d_q, ctx->d_D1, nl, ctx->k, ctx->h, M, Up);
      boundary_gather(s, X, ctx->d_D1, ctx->nL, ctx->h, M, ub, psib);
      scattered_data(s, ub, psib, ui, dni, (long long)nbM, PS);
      if (emu) {
        oz_slice_wide(s, re_view_t(PS, M, 0), M, 2 * nb, false, ozs);
        oz_slice_wide(s, re_view_t(PS, M, 1), M, 2 * nb, false, ozs + ob_ps);
        const cudaError_t e = oz_zmul_wide(s, nb, M, 2 * nb, ctx->d_ds_oz, ctx->d_ds_oz + ob_ds, ozs, ozs + ob_ps,
                                           -1.0, 0.0, rext, M, ozp);
        if (e != cudaSuccess) return fail(ctx, HS_ECUDA, std::string("emulated FP64 product: ") + cudaGetErrorString(e));
      } else {
        gemm<double2, double2, double2>(s, OP_N, OP_N, nb, M, 2 * nb, mone, ctx->d_DS, 2 * nb, 0, PS, M, 0, zero,
                                        rext, M, 0, 1);
      }
    }
    // The rest of the pass is FP32 work on fixed buffers: replayed from a
    // captured graph (one for the first pass, one for the corrections).
    const bool first = it == 0;
    auto body = [&]() -> int {
      if (first) {
        // exterior right-hand side (D - I/2) u_inc - S d_n u_inc, in FP32 (the
        // first pass is an FP32 solve; the corrections use FP64 residuals)
        convert_d2f(s, ui, PS32, (long long)nbM);
        convert_d2f(s, dni, PS32 + nbM, (long long)nbM);
        gemm<float2, float2, float2>(s, OP_N, OP_N, nb, M, 2 * nb, fone, ctx->d_DS32, 2 * nb, 0, PS32, M, 0, fzero,
                                     f32, M, 0, 1);
      } else {
        convert_d2f(s, rext, r32, (long long)nbM);
        // FP32 correction: particular leaf solutions, upward pass, root
        leaf_particular(s, ctx->ws32, nl, ctx->d_k, M, Up, B0, tmp, wtmp);
        float2 *Hc = B0, *Hp = B1;
        for (int li = 0; li < nlev; ++li) {
          residual_iface(s, ctx->levels[li], X, ctx->d_D1, ctx->nL, ctx->h, ctx->d_k, M, S3);
          sweep_up_level<float2>(s, ctx->levels[li], ctx->ops32[li], Hc, S3, TT[li], Hp, M);
          std::swap(Hc, Hp);
        }
        permute_rows<float2>(s, Hc, ctx->d_root_of_bie, nb, M, tmp);  // root h in boundary-node order
        CK(cudaMemcpyAsync(f32, r32, sizeof(float2) * nbM, cudaMemcpyDeviceToDevice, s));
        gemm<float2, float2, float2>(s, OP_N, OP_N, nb, M, nb, fone, ctx->d_B2_32, nb, 0, tmp, M, 0, fone, f32, M, 0,
                                     1);
      }
      gemm<float2, float2, float2>(s, OP_N, OP_N, nb, M, nb, fone, ctx->d_Rb32, nb, 0, f32, M, 0, fzero, r32, M, 0, 1);
      // downward sweep (adds the particular interface impedances after the first pass)
      permute_rows<float2>(s, r32, ctx->d_bie_of_root, nb, M, B1);  // root box order
      const float2* Fp = B1;
      float2* out = B0;
      for (int li = nlev - 1; li >= 0; --li) {
        sweep_down_level<float2>(s, ctx->levels[li], ctx->ops32[li], Fp, TT[li], out, M, !first);
        Fp = out;
        out = (out == B0) ? B1 : B0;
      }
      gemm<float2, float2, float2>(s, OP_N, OP_N, NL, M, NE, fone, ctx->d_Y32, NE, (long long)NL * NE, Fp, M,
                                   (long long)NE * M, first ? fzero : fone, Up, M, (long long)NL * M, nl);
      convert_f2d_add(s, Up, X, (long long)nX);
      // far field of this pass's FP32 field (the solution on the first pass, the
      // correction after it), in FP32: its norm relative to the first pass's far
      // field is the relative change of the far field
      scattered32(s, Up, ctx->d_D1, ctx->nL, ctx->h, M, ui, dni, first, PS32);
      gemm<float2, float2, float2>(s, OP_T, OP_T, M, P, 2 * nb, fone, PS32, M, 0, A2_32, 2 * nb, 0, fzero, duf, P, 0,
                                   1);
      CK(cudaMemsetAsync(nrm, 0, sizeof(double), s));
      norm2_32(s, duf, (long long)M * P, nrm);
      return HS_OK;
    };
    const bool capture = g_use_graphs && !prof_active(2) && !prof_active(3);
    // keyed by the buffers and the sizes only: the body's kernels read k on the device
    CKR(run_captured(ctx, s, ctx->pgraph[first ? 0 : 1], capture, ui, M, P, 0.0, body));
    double dn2 = 0.0;
    CK(cudaMemcpyAsync(&dn2, nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ctx->refine_iters = it + 1;
    if (it == 0) {
      uf0_n2 = dn2;
    } else {
      const double upd = uf0_n2 > 0 ? std::sqrt(dn2 / uf0_n2) : 0.0;
      // error of the new iterate: the update itself until the contraction
      // rate rho of the passes is observed, then upd * rho / (1 - rho)
      double est = upd;
      if (prev_upd > 0.0 && upd < 0.5 * prev_upd) {
        const double rho = upd / prev_upd;
        est = upd * rho / (1.0 - rho);
      }
      ctx->refine_update = upd;
      ctx->refine_est = est;
      prev_upd = upd;
      if (est <= tol) {
        converged = true;
        break;
      }
    }
  }
  CK(cudaGetLastError());
  if (tc_timed_out(s)) return fail(ctx, HS_ETIMEOUT, "a tensor-core GEMM wait gave up");
  if (!converged) return fail(ctx, HS_ENOCONV, "iterative refinement did not reach the tolerance");
  if (ufar) {  // far field of the converged FP64 iterate, in FP64
    boundary_gather(s, X, ctx->d_D1, ctx->nL, ctx->h, M, ub, psib);
    scattered_data(s, ub, psib, ui, dni, (long long)nbM, PS);
    if (emu) {  // uf = PS^T A2^T
      char *pa = ozs, *pb = ozs + 2 * ob_psa;
      oz_slice_wide(s, re_view_t(PS, M, 0), M, 2 * nb, true, pa);
      oz_slice_wide(s, re_view_t(PS, M, 1), M, 2 * nb, true, pa + ob_psa);
      oz_slice_wide(s, re_view(A2, 2 * nb, 0), P, 2 * nb, false, pb);
      oz_slice_wide(s, re_view(A2, 2 * nb, 1), P, 2 * nb, false, pb + ob_a2);
      const cudaError_t e =
          oz_zmul_wide(s, M, P, 2 * nb, pa, pa + ob_psa, pb, pb + ob_a2, 1.0, 0.0, uf, P, ozp);
      if (e != cudaSuccess) return fail(ctx, HS_ECUDA, std::string("emulated FP64 product: ") + cudaGetErrorString(e));
    } else {
      gemm<double2, double2, double2>(s, OP_T, OP_T, M, P, 2 * nb, one, PS, M, 0, A2, 2 * nb, 0, zero, uf, P, 0, 1);
    }
  }
  if (ufar) CK(cudaMemcpyAsync(ufar, uf, sizeof(double2) * M * P, cudaMemcpyDeviceToDevice, s));
  if (Xout) CK(cudaMemcpyAsync(Xout, X, sizeof(double2) * nX, cudaMemcpyDeviceToDevice, s));
  return HS_OK;
}

// Forward fields on the interior grid (Ug, M x n14 x n14) and adjoint fields
// (Zg, P x n14 x n14); workspace carved from `a` after `reserve` bytes.
int fields_and_adjoint(hs_ctx* ctx, cudaStream_t s, const double* alphas, int M, const double* thetas, int P,
                       double2* Ug, double2* Zg, Arena& a) {
  const int nb = ctx->B.nb;
  const int nr = std::max(M, P);
  double2 *ui = a.get<double2>((size_t)nb * M), *dni = a.get<double2>((size_t)nb * M);
  double2 *f = a.get<double2>((size_t)nb * M), *g = a.get<double2>((size_t)nb * M);
  double2 *bufA = a.get<double2>(field_buf_elems(ctx, nr)), *bufB = a.get<double2>(field_buf_elems(ctx, nr));
  double2* T3 = a.get<double2>(t3_elems(ctx, nr));
  double2* Uleaf = a.get<double2>((size_t)ctx->nleaf * NL * nr);
  double2* A2 = a.get<double2>((size_t)P * 2 * nb);
  double2 *E = a.get<double2>((size_t)nb * P), *CP = a.get<double2>((size_t)nb * P);
  if (a.over) return fail(ctx, HS_ENOMEM, "workspace request beyond its sizing");
  CKR(root_solve(ctx, s, alphas, M, ui, dni, f, g));
  CKR(sweep_down(ctx, s, f, M, bufA, bufB, T3, Uleaf));
  leaf_to_grid(s, Uleaf, NL, ctx->nL, M, Ug);
  farfield_matrix(s, ctx->B, ctx->k, ctx->cfg.R, thetas, P, A2);
  CKR(sweep_adjoint(ctx, s, A2, P, E, CP, bufA, bufB, T3, Uleaf));
  leaf_to_grid(s, Uleaf, NI, ctx->nL, P, Zg);
  return HS_OK;
}

size_t fields_and_adjoint_bytes(hs_ctx* ctx, int M, int P) {
  const int nb = ctx->B.nb;
  const int nr = std::max(M, P);
  return 4 * Arena::bytes((size_t)nb * M, 16) + 2 * Arena::bytes(field_buf_elems(ctx, nr), 16) +
         Arena::bytes(t3_elems(ctx, nr), 16) + Arena::bytes((size_t)ctx->nleaf * NL * nr, 16) +
         Arena::bytes((size_t)P * 2 * nb, 16) + 2 * Arena::bytes((size_t)nb * P, 16);
}


size_t mixed_adjoint_bytes(hs_ctx* ctx, int P) {
  const size_t nb = ctx->B.nb, nl = ctx->nleaf;
  size_t b = Arena::bytes(nl * NL * P, 8) + 2 * Arena::bytes(field_buf_elems(ctx, P), 8) +
             3 * Arena::bytes(nb * P, 8) + Arena::bytes(nl * NI * P, 8) + Arena::bytes(nl * NE * P, 8) +
             Arena::bytes((size_t)ctx->if_rows * P, 16) + Arena::bytes(nb * P, 16) + Arena::bytes(2 * nb * P, 16) +
             Arena::bytes(8, 8);
  for (auto& L : ctx->levels) b += Arena::bytes((size_t)L.nbox * 2 * L.ni * P, 8);
  if (g_oz_enabled)
    b += Arena::bytes(2 * oz_wide_bytes(P, (int)nb, false), 1) + Arena::bytes(4 * oz_partial_bytes(2 * (int)nb, P, (int)nb), 1);
  return b;
}

// Mixed precision: the adjoint fields Z = A^{-T} L of the receiver functionals
// (Theorem 3.2's w_p, discretely: L_p reads u_far(p) = A2[p] . [u; d_n u] on
// the boundary) at every interior leaf node, FP64-accurate, by iterative
// refinement in the row space of the discrete system: each pass computes the
// FP64 residual L - A^T Y of every unknown (adjoint_residual: the transposed
// PDE, interface and exterior rows) and solves the transposed FP32 system for
// the correction.  That FP32 solve is the exact transpose of the forward
// correction solve of mixed_solve, step by step in reverse order:
//   leaf solution operators        lambda = Y32^T g
//   downward sweep (transposed)    per level from the leaves up: MU = interface
//                                  part of the children's lambda, parent
//                                  lambda = exterior part + [X; Z]^T MU
//   root                           Yext = C^{-T} lambda_root (C^{-1} kept
//                                  explicitly), root h-adjoint = B2^T Yext
//   upward pass (transposed)       per level from the root down (MU preloaded),
//                                  giving the s_a, s_b adjoints of that level
//   leaf particular (transposed)   Ypde = A_ii^{-T} (g_i + N_i^T (-K^{-T}
//                                  (g_e - X^T g_i - 2 i eta h-adjoint)))
// Stops like the forward refinement, on the relative change of Ypde (the
// adjoint the Jacobian and the gradient use): once two changes give the
// contraction rate rho, the error estimate is the change times rho / (1 - rho).
// Z64: [leaf][196][P] (FP64, output).  A2: [P][2 nb] FP64.
// With refine == false one pass (the FP32 transposed solve of L) is returned:
// for products that carry FP32 rounding anyway (the explicit FP32 Jacobian).
// passes: 0 = refine to refine_tol (HS_ENOCONV after refine_max_iter passes);
// n > 0 = exactly n passes (the FP32 solve and n - 1 FP64-residual corrections).
int mixed_adjoint(hs_ctx* ctx, cudaStream_t s, const double2* A2, int P, double2* Z64, Arena& a, int passes = 0) {
  const int nb = ctx->B.nb, nl = ctx->nleaf, nlev = (int)ctx->levels.size();
  const size_t nbP = (size_t)nb * P;
  const double eta = ctx->k;
  const double tol = ctx->cfg.refine_tol > 0 ? ctx->cfg.refine_tol : 1e-9;
  const bool refine = passes != 1;
  const int max_iter = passes > 0 ? passes : ctx->cfg.refine_max_iter > 0 ? ctx->cfg.refine_max_iter : 8;
  const float2 one = make_float2(1.f, 0.f), mone = make_float2(-1.f, 0.f), zero = make_float2(0.f, 0.f);
  float2* G = a.get<float2>((size_t)nl * NL * P);
  float2 *bufA = a.get<float2>(field_buf_elems(ctx, P)), *bufB = a.get<float2>(field_buf_elems(ctx, P));
  float2 *r32 = a.get<float2>(nbP), *f32 = a.get<float2>(nbP), *t32 = a.get<float2>(nbP);
  float2* dY = a.get<float2>((size_t)nl * NI * P);
  float2* tE = a.get<float2>((size_t)nl * NE * P);
  double2* Yif = a.get<double2>((size_t)ctx->if_rows * P);
  double2* Yext = a.get<double2>(nbP);
  double2* V = a.get<double2>(2 * nbP);
  double* nrm = a.get<double>(8);
  std::vector<float2*> MU(nlev);
  for (int li = 0; li < nlev; ++li) MU[li] = a.get<float2>((size_t)ctx->levels[li].nbox * 2 * ctx->levels[li].ni * P);
  // the exterior rows' transposed product DS^T Yext by the emulated FP64 product:
  // DS^T sliced once per k, Yext (as the right operand) once per pass
  const bool emu = g_oz_enabled;
  const size_t ob_y = emu ? oz_wide_bytes(P, nb, false) : 0, ob_part = emu ? oz_partial_bytes(2 * nb, P, nb) : 0;
  char* ozs = emu ? a.get<char>(2 * ob_y) : nullptr;
  char* ozp = emu ? a.get<char>(4 * ob_part) : nullptr;
  if (a.over) return fail(ctx, HS_ENOMEM, "workspace request beyond its sizing");
  const size_t ob_dst = oz_wide_bytes(2 * nb, nb, true);
  if (emu && ctx->dst_oz_k != ctx->bie_k) {
    if (!ctx->d_dst_oz) CKR(dalloc(ctx, &ctx->d_dst_oz, 2 * ob_dst));
    oz_slice_wide(s, re_view_t(ctx->d_DS, 2 * nb, 0), 2 * nb, nb, true, ctx->d_dst_oz);
    oz_slice_wide(s, re_view_t(ctx->d_DS, 2 * nb, 1), 2 * nb, nb, true, ctx->d_dst_oz + ob_dst);
    ctx->dst_oz_k = ctx->bie_k;
  }
  const LeafScratchT<float>& w = ctx->ws32;
  const long long sG = (long long)NL * P;
  Phase ph("hs_adjoint_refine");
  CK(cudaMemsetAsync(Z64, 0, sizeof(double2) * (size_t)nl * NI * P, s));
  if (ctx->if_rows > 0) CK(cudaMemsetAsync(Yif, 0, sizeof(double2) * (size_t)ctx->if_rows * P, s));
  CK(cudaMemsetAsync(Yext, 0, sizeof(double2) * nbP, s));
  ctx->adj_iters = 0;
  ctx->adj_update = -1.0;
  ctx->adj_est = -1.0;
  double prev_upd = 0.0, y0_n2 = 0.0;
  bool converged = false;
  for (int it = 0; it < max_iter; ++it) {
    Phase pp("hs_adjoint_pass");
    const bool first = it == 0;
    // FP64 residual L - A^T Y of every unknown (L itself on the first pass)
    if (!first && emu) {
      oz_slice_wide(s, re_view_t(Yext, P, 0), P, nb, false, ozs);
      oz_slice_wide(s, re_view_t(Yext, P, 1), P, nb, false, ozs + ob_y);
      const cudaError_t e = oz_zmul_wide(s, 2 * nb, P, nb, ctx->d_dst_oz, ctx->d_dst_oz + ob_dst, ozs, ozs + ob_y, 1.0,
                                         0.0, V, P, ozp);
      if (e != cudaSuccess) return fail(ctx, HS_ECUDA, std::string("emulated FP64 product: ") + cudaGetErrorString(e));
    } else if (!first) {
      gemm<double2, double2, double2>(s, OP_T, OP_N, 2 * nb, P, nb, make_double2(1, 0), ctx->d_DS, 2 * nb, 0, Yext, P,
                                      0, make_double2(0, 0), V, P, 0, 1);
    }
    adjoint_residual(s, Z64, ctx->d_adj_desc, Yif, A2, first ? nullptr : V, ctx->d_q, ctx->d_D1, nl, nb, ctx->k,
                     ctx->h, eta, P, first, G);
    // transposed FP32 solve: leaf solution operators, then the transposed
    // downward sweep from the leaves to the root
    gemm<float2, float2, float2>(s, OP_T, OP_N, NE, P, NL, one, ctx->d_Y32, NE, (long long)NL * NE, G, P, sG, zero,
                                 bufA, P, (long long)NE * P, nl);
    float2 *Lc = bufA, *Lp = bufB;
    for (int li = 0; li < nlev; ++li) {
      sweep_adjoint_up_level<float2>(s, ctx->levels[li], ctx->ops32[li], Lc, MU[li], Lp, P);
      std::swap(Lc, Lp);
    }
    // root (boundary-node order): Yext = C^{-T} lambda, h-adjoint = B2^T Yext
    permute_rows<float2>(s, Lc, ctx->d_root_of_bie, nb, P, r32);
    gemm<float2, float2, float2>(s, OP_T, OP_N, nb, P, nb, one, ctx->d_Rb32, nb, 0, r32, P, 0, zero, f32, P, 0, 1);
    gemm<float2, float2, float2>(s, OP_T, OP_N, nb, P, nb, one, ctx->d_B2_32, nb, 0, f32, P, 0, zero, t32, P, 0, 1);
    permute_rows<float2>(s, t32, ctx->d_bie_of_root, nb, P, Lp);
    std::swap(Lc, Lp);  // Lc: the root's h-adjoint in root box order
    // transposed upward pass from the root to the leaves
    for (int li = nlev - 1; li >= 0; --li) {
      sweep_adjoint_level<float2>(s, ctx->levels[li], ctx->ops32[li], Lc, MU[li], Lp, P, true, true);
      iface_adj_add(s, MU[li], ctx->levels[li].nbox, ctx->levels[li].ni, P, Yif + ctx->if_off[li] * P);
      std::swap(Lc, Lp);
    }
    // transposed leaf particular solve (Lc: every leaf's h-adjoint)
    if (w.P) {  // impedance-form leaves: the interior rows of L^{-T} [g_i; g_e] are P^T [g_i; g_e]
      leaf_hadj(s, Lc, nl, eta, P, G);
      gemm<float2, float2, float2>(s, OP_T, OP_N, NI, P, NL, one, w.P, NI, (long long)NL * NI, G, P, sG, zero, dY, P,
                                   (long long)NI * P, nl);
    } else {
      gemm<float, float2, float2>(s, OP_T, OP_N, NE, P, NI, mone, w.Aie, NE, (long long)NI * NE, G, P, sG, one,
                                  G + (long long)NI * P, P, sG, nl);
      leaf_hadj(s, Lc, nl, eta, P, G);
      gemm<float2, float2, float2>(s, OP_T, OP_N, NE, P, NE, mone, w.Kinv, NE, (long long)NE * NE,
                                   G + (long long)NI * P, P, sG, zero, tE, P, (long long)NE * P, nl);
      gemm<float, float2, float2>(s, OP_T, OP_N, NI, P, NE, one, w.Ni, NI, (long long)NE * NI, tE, P,
                                  (long long)NE * P, one, G, P, sG, nl);
      gemm<float, float2, float2>(s, OP_T, OP_N, NI, P, NI, one, w.Ainv, NI, (long long)NI * NI, G, P, sG, zero, dY,
                                  P, (long long)NI * P, nl);
    }
    // accumulate in FP64; the change of Ypde is the stopping quantity
    convert_f2d_add(s, dY, Z64, (long long)nl * NI * P);
    convert_f2d_add(s, f32, Yext, (long long)nbP);
    CK(cudaMemsetAsync(nrm, 0, sizeof(double), s));
    norm2_32(s, dY, (long long)nl * NI * P, nrm);
    double dn2 = 0.0;
    CK(cudaMemcpyAsync(&dn2, nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ctx->adj_iters = it + 1;
    if (first) {
      y0_n2 = dn2;
      if (!(y0_n2 > 0.0) || !refine) {  // no receiver sees the interior (Z = 0 exactly), or one pass asked for
        converged = true;
        break;
      }
    } else {
      const double upd = std::sqrt(dn2 / y0_n2);
      double est = upd;
      if (prev_upd > 0.0 && upd < 0.5 * prev_upd) {
        const double rho = upd / prev_upd;
        est = upd * rho / (1.0 - rho);
      }
      ctx->adj_update = upd;
      ctx->adj_est = est;
      prev_upd = upd;
      if (est <= tol || (passes > 0 && it + 1 == passes)) {
        converged = true;
        break;
      }
    }
  }
  CK(cudaGetLastError());
  if (tc_timed_out(s)) return fail(ctx, HS_ETIMEOUT, "a tensor-core GEMM wait gave up");
  if (!converged) return fail(ctx, HS_ENOCONV, "adjoint refinement did not reach the tolerance");
  return HS_OK;
}

size_t mixed_fields_bytes(hs_ctx* ctx, int M, int P) {
  const int nb = ctx->B.nb;
  return Arena::bytes((size_t)ctx->nleaf * NL * M, 16) + Arena::bytes((size_t)P * 2 * nb, 16) +
         Arena::bytes((size_t)ctx->nleaf * NI * P, 16) +
         std::max(mixed_bytes(ctx, M, P), mixed_adjoint_bytes(ctx, P));
}

// Mixed precision: far field F and forward fields Ug from the refined forward
// solve, adjoint fields Zg from the refined adjoint solve (both FP64-accurate),
// on the interior grid.
int mixed_fields_and_adjoint(hs_ctx* ctx, cudaStream_t s, const double* alphas, int M, const double* thetas, int P,
                             double2* F, double2* Ug, double2* Zg, Arena& a, int adjoint_passes = 0) {
  const int nb = ctx->B.nb;
  double2* X = a.get<double2>((size_t)ctx->nleaf * NL * M);
  double2* A2 = a.get<double2>((size_t)P * 2 * nb);
  double2* Z64 = a.get<double2>((size_t)ctx->nleaf * NI * P);
  if (a.over) return fail(ctx, HS_ENOMEM, "workspace request beyond its sizing");
  {
    Arena sub = a;
    CKR(mixed_solve(ctx, s, alphas, M, thetas, P, F, X, sub));
  }
  leaf_to_grid(s, X, NL, ctx->nL, M, Ug);
  farfield_matrix(s, ctx->B, ctx->k, ctx->cfg.R, thetas, P, A2);
  {
    Arena sub = a;
    CKR(mixed_adjoint(ctx, s, A2, P, Z64, sub, adjoint_passes));
  }
  leaf_to_grid(s, Z64, NI, ctx->nL, P, Zg);
  CK(cudaGetLastError());
  return HS_OK;
}

// Mixed precision: J from the refined forward fields and the refined adjoint
// fields (both FP64-accurate), contracted in FP64 like the FP64 context's.
// F (optional, M x P) receives the refined far field of the same solve.
int jacobian_into_mixed(hs_ctx* ctx, cudaStream_t s, const double* alphas, int M, const double* thetas, int P,
                        double2* J, Arena& a, double2* F_out = nullptr) {
  const int nX = ctx->n14, S1 = ctx->S1, S2 = ctx->S2;
  const size_t plane = (size_t)nX * nX, MP = (size_t)M * P;
  const int C = contract_chunk(M, P, nX, S1, g_contract_budget);
  double2* Ug = a.get<double2>(plane * M);
  double2* Zg = a.get<double2>(plane * P);
  double2* F = a.get<double2>(MP);
  if (a.over) return fail(ctx, HS_ENOMEM, "workspace request beyond its sizing");
  {
    Arena sub = a;
    CKR(mixed_fields_and_adjoint(ctx, s, alphas, M, thetas, P, F, Ug, Zg, sub));
  }
  if (F_out) CK(cudaMemcpyAsync(F_out, F, sizeof(double2) * MP, cudaMemcpyDeviceToDevice, s));
  double2* W = a.get<double2>(plane * C);
  double2* T = a.get<double2>((size_t)nX * S1 * C);
  const size_t ozb = g_oz_enabled ? contract_emulated_bytes(C, nX, S1, S2) : 0;
  char* oz = ozb ? a.get<char>(ozb) : nullptr;
  if (a.over) return fail(ctx, HS_ENOMEM, "workspace request beyond its sizing");
  interior_sine_tables(s, ctx->d_xint, nX, S1, S2, ctx->d_sxi, ctx->d_syi);
  Phase ph("hs_jacobian_contract");
  contract_jacobian(s, Ug, Zg, M, P, nX, ctx->d_sxi, ctx->d_syi, S1, S2, ctx->k * ctx->k, J, W, T, C, oz, ozb);
  CK(cudaGetLastError());
  return HS_OK;
}

size_t jacobian_bytes_mixed(hs_ctx* ctx, int M, int P) {
  const int nX = ctx->n14;
  const size_t plane = (size_t)nX * nX, MP = (size_t)M * P;
  const int C = contract_chunk(M, P, nX, ctx->S1, g_contract_budget);
  const size_t ozb = g_oz_enabled ? contract_emulated_bytes(C, nX, ctx->S1, ctx->S2) : 0;
  return Arena::bytes(plane * M, 16) + Arena::bytes(plane * P, 16) + Arena::bytes(MP, 16) +
         std::max(mixed_fields_bytes(ctx, M, P),
                  Arena::bytes(plane * C, 16) + Arena::bytes((size_t)nX * ctx->S1 * C, 16) + Arena::bytes(ozb, 1));
}

int jacobian_into(hs_ctx* ctx, cudaStream_t s, const double* alphas, int M, const double* thetas, int P, double2* J,
                  Arena& a) {
  if (ctx->cfg.precision == HS_MIXED) return jacobian_into_mixed(ctx, s, alphas, M, thetas, P, J, a);
  const size_t plane = (size_t)ctx->n14 * ctx->n14;
  const int C = contract_chunk(M, P, ctx->n14, ctx->S1, g_contract_budget);
  double2* Ug = a.get<double2>(plane * M);
  double2* Zg = a.get<double2>(plane * P);
  if (a.over) return fail(ctx, HS_ENOMEM, "workspace request beyond its sizing");
  {
    Arena sub = a;  // the solves' scratch is reused by the contraction afterwards (same stream)
    CKR(fields_and_adjoint(ctx, s, alphas, M, thetas, P, Ug, Zg, sub));
  }
  double2* W = a.get<double2>(plane * C);
  double2* T = a.get<double2>((size_t)ctx->n14 * ctx->S1 * C);
  const size_t ozb = g_oz_enabled ? contract_emulated_bytes(C, ctx->n14, ctx->S1, ctx->S2) : 0;
  char* oz = ozb ? a.get<char>(ozb) : nullptr;
  if (a.over) return fail(ctx, HS_ENOMEM, "workspace request beyond its sizing");
  interior_sine_tables(s, ctx->d_xint, ctx->n14, ctx->S1, ctx->S2, ctx->d_sxi, ctx->d_syi);
  Phase ph("hs_jacobian_contract");
  contract_jacobian(s, Ug, Zg, M, P, ctx->n14, ctx->d_sxi, ctx->d_syi, ctx->S1, ctx->S2, ctx->k * ctx->k, J, W, T, C,
                    oz, ozb);
  CK(cudaGetLastError());
  return HS_OK;
}

size_t jacobian_bytes(hs_ctx* ctx, int M, int P) {
  if (ctx->cfg.precision == HS_MIXED) return jacobian_bytes_mixed(ctx, M, P);
  const size_t plane = (size_t)ctx->n14 * ctx->n14;
  const int C = contract_chunk(M, P, ctx->n14, ctx->S1, g_contract_budget);
  const size_t ozb = g_oz_enabled ? contract_emulated_bytes(C, ctx->n14, ctx->S1, ctx->S2) : 0;
  return Arena::bytes(plane * M, 16) + Arena::bytes(plane * P, 16) +
         std::max(Arena::bytes(plane * C, 16) + Arena::bytes((size_t)ctx->n14 * ctx->S1 * C, 16) +
                      Arena::bytes(ozb, 1),
                  fields_and_adjoint_bytes(ctx, M, P));
}

int need_fp64(hs_ctx* ctx) {
  if (ctx->cfg.precision != HS_FP64) return fail(ctx, HS_EINVAL, "this call needs a context created with HS_FP64");
  return HS_OK;
}

int valid_angles(hs_ctx* ctx, int M, int P) {
  if (M <= 0 || P <= 0 || M > 65535 || P > 65535) return fail(ctx, HS_EINVAL, "M and P must be in 1..65535");
  return HS_OK;
}

// grad = Re J^H (F - data) = k^2 Re sum_x s_m1 s_m2 sum_d u_d(x) sum_p conj(F - data)_dp z_p(x)
int gradient_core(hs_ctx* ctx, cudaStream_t s, const double* ddata, const double* da, int M, const double* dt,
                         int P, double* dgrad, double* dmis, Arena& a) {
  const int MP = M * P;
  const size_t plane = (size_t)ctx->n14 * ctx->n14;
  double2* F = a.get<double2>(MP);
  double2* res = a.get<double2>(MP);
  double2* Ug = a.get<double2>(plane * M);
  double2* Zg = a.get<double2>(plane * P);
  double2* Zmix = a.get<double2>(plane * M);
  double* hre = a.get<double>(plane);
  double* T1 = a.get<double>((size_t)ctx->S1 * ctx->n14);
  if (a.over) return fail(ctx, HS_ENOMEM, "workspace request beyond its sizing");
  const bool mixed = ctx->cfg.precision == HS_MIXED;
  if (mixed) {  // refined far field and forward fields, FP32 adjoint fields
    Arena sub = a;
    CKR(mixed_fields_and_adjoint(ctx, s, da, M, dt, P, F, Ug, Zg, sub));
  } else {
    Arena sub = a;
    const int nb = ctx->B.nb;
    double2 *ui = sub.get<double2>((size_t)nb * M), *dni = sub.get<double2>((size_t)nb * M);
    double2 *f = sub.get<double2>((size_t)nb * M), *g = sub.get<double2>((size_t)nb * M);
    double2* PS = sub.get<double2>((size_t)2 * nb * M);
    double2* A2 = sub.get<double2>((size_t)P * 2 * nb);
    CKR(root_solve(ctx, s, da, M, ui, dni, f, g));
    boundary_data(s, nb, M, ctx->k, f, g, ui, dni, PS);
    farfield_matrix(s, ctx->B, ctx->k, ctx->cfg.R, dt, P, A2);
    gemm<double2, double2, double2>(s, OP_T, OP_T, M, P, 2 * nb, make_double2(1, 0), PS, M, 0, A2, 2 * nb, 0,
                                    make_double2(0, 0), F, P, 0, 1);
  }
  CK(cudaMemsetAsync(dmis, 0, sizeof(double), s));
  residual(s, ddata, F, MP, res, nullptr, dmis);  // res = data - F
  if (!mixed) CKR(fields_and_adjoint(ctx, s, da, M, dt, P, Ug, Zg, a));
  // Zmix = conj(F - data) Zg = -conj(res) Zg  (M x plane)
  conj_neg(s, res, MP);
  gemm<double2, double2, double2>(s, OP_N, OP_N, M, (int)plane, P, make_double2(1, 0), res, P, 0, Zg, (int)plane, 0,
                                  make_double2(0, 0), Zmix, (int)plane, 0, 1);
  gradient_combine(s, Ug, Zmix, M, (long long)plane, hre);
  interior_sine_tables(s, ctx->d_xint, ctx->n14, ctx->S1, ctx->S2, ctx->d_sxi, ctx->d_syi);
  // T1 = sx hre^T  (S1 x nY);  grad = k^2 T1 sy^T
  gemm<double, double, double>(s, OP_N, OP_T, ctx->S1, ctx->n14, ctx->n14, 1.0, ctx->d_sxi, ctx->n14, 0, hre,
                               ctx->n14, 0, 0.0, T1, ctx->n14, 0, 1);
  gemm<double, double, double>(s, OP_N, OP_T, ctx->S1, ctx->S2, ctx->n14, ctx->k * ctx->k, T1, ctx->n14, 0,
                               ctx->d_syi, ctx->n14, 0, 0.0, dgrad, ctx->S2, 0, 1);
  half_in_place(s, dmis);
  CK(cudaGetLastError());
  return HS_OK;
}

size_t gradient_bytes(hs_ctx* ctx, int M, int P) {
  const int MP = M * P;
  const size_t plane = (size_t)ctx->n14 * ctx->n14;
  return 2 * Arena::bytes(MP, 16) + Arena::bytes(plane * M, 16) * 2 + Arena::bytes(plane * P, 16) +
         Arena::bytes(plane, 8) + Arena::bytes((size_t)ctx->S1 * ctx->n14, 8) +
         (ctx->cfg.precision == HS_MIXED ? mixed_fields_bytes(ctx, M, P) : fields_and_adjoint_bytes(ctx, M, P));
}

}  // namespace

namespace hs {

// CUDA device ordinal the context works on.
int ctx_device(const hs_ctx* ctx) { return ctx->cfg.device; }

// Bytes of caller-provided scratch a far-field solve of M incidences and P
// receivers needs (see solve_far_in_scratch).
size_t far_solve_scratch_bytes(const hs_ctx* ctx, int M, int P) {
  const size_t nb = (size_t)ctx->B.nb;
  return 16 * nb * (6 * (size_t)M + 2 * (size_t)P);
}

// The far-field solve of solve_into with every temporary carved from the
// caller's scratch (no allocation).  Used by the allocation-free entry point.
int solve_far_in_scratch(hs_ctx* ctx, void* stream, const double* alphas, int M, const double* thetas, int P,
                         double* ufar, void* scratch, size_t scratch_bytes) {
  CKR(check_ctx(ctx, true));
  LaunchScope ls(ctx);
  CKR(need_fp64(ctx));
  CKR(valid_angles(ctx, M, P));
  if (!alphas || !thetas || !ufar || !scratch) return fail(ctx, HS_EINVAL, "NULL pointer");
  if (far_solve_scratch_bytes(ctx, M, P) > scratch_bytes)
    return fail(ctx, HS_EINVAL, "M and P too large for the fixed scratch: need 16*N_b*(6M+2P) = " +
                                    std::to_string(far_solve_scratch_bytes(ctx, M, P)) + " bytes, have " +
                                    std::to_string(scratch_bytes));
  cudaStream_t s = pick(ctx, stream);
  const size_t nb = (size_t)ctx->B.nb;
  double2* p = reinterpret_cast<double2*>(scratch);
  double2 *ui = p, *dni = ui + nb * M, *f = dni + nb * M, *g = f + nb * M;
  double2 *PS = g + nb * M, *A2 = PS + 2 * nb * M;
  CKR(root_solve(ctx, s, alphas, M, ui, dni, f, g));
  boundary_data(s, (int)nb, M, ctx->k, f, g, ui, dni, PS);
  farfield_matrix(s, ctx->B, ctx->k, ctx->cfg.R, thetas, P, A2);
  gemm<double2, double2, double2>(s, OP_T, OP_T, M, P, 2 * (int)nb, make_double2(1, 0), PS, M, 0, A2, 2 * (int)nb, 0,
                                  make_double2(0, 0), reinterpret_cast<double2*>(ufar), P, 0, 1);
  CK(cudaGetLastError());
  return HS_OK;
}

}  // namespace hs

// ============================== C ABI =====================================
extern "C" {

int hs_create(hs_ctx** out, const hs_config* cfg) {
  if (!out || !cfg) return HS_EINVAL;
  *out = nullptr;
  const int nL = cfg->leaves_per_side;
  if (nL < 1 || nL > 256 || (nL & (nL - 1)) != 0) return HS_EINVAL;
  if (cfg->S1 < 1 || cfg->S2 < 1 || cfg->S1 > 512 || cfg->S2 > 512) return HS_EINVAL;
  if (!(cfg->R > std::sqrt(2.0))) return HS_EINVAL;
  if (cfg->precision != HS_FP64 && cfg->precision != HS_MIXED) return HS_EINVAL;
  if (!(cfg->bm_eta >= 0.0) || !std::isfinite(cfg->bm_eta)) return HS_EINVAL;
  if (cfg->leaf_impedance != 0 && cfg->leaf_impedance != 1) return HS_EINVAL;
  hs_ctx* ctx = new (std::nothrow) hs_ctx();
  if (!ctx) return HS_ENOMEM;
  ctx->cfg = *cfg;
  ctx->nL = nL;
  ctx->S1 = cfg->S1;
  ctx->S2 = cfg->S2;
  LaunchScope ls(ctx);
  cudaError_t e = cudaSetDevice(cfg->device);
  if (e != cudaSuccess) {
    delete ctx;
    return HS_ECUDA;
  }
  if (cfg->stream) {
    ctx->stream = (cudaStream_t)cfg->stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return HS_ECUDA;
    }
    ctx->own_stream = true;
  }
  int r = setup(ctx);
  if (r != HS_OK) {
    hs_destroy(ctx);
    return r;
  }
  *out = ctx;
  return HS_OK;
}

int hs_node_coords(const hs_ctx* ctx, double* x, double* y) {
  if (!ctx || !x || !y) return HS_EINVAL;
  std::vector<double> t = lobatto(16);
  const int nL = ctx->nL;
  for (int leaf = 0; leaf < nL * nL; ++leaf) {
    int ix = leaf % nL, iy = leaf / nL;
    for (int a = 0; a < 16; ++a)
      for (int b = 0; b < 16; ++b) {
        size_t i = ((size_t)leaf * 16 + a) * 16 + b;
        x[i] = -1.0 + ix * ctx->h + (t[a] + 1.0) * ctx->h / 2.0;
        y[i] = -1.0 + iy * ctx->h + (t[b] + 1.0) * ctx->h / 2.0;
      }
  }
  return HS_OK;
}

int hs_build(hs_ctx* ctx, const double* c, int S1, int S2, double k) {
  CKR(check_ctx(ctx, false));
  LaunchScope ls(ctx);
  if (!c || S1 != ctx->S1 || S2 != ctx->S2) return fail(ctx, HS_EINVAL, "coefficient shape must be S1 x S2 of the config");
  if (!(k > 0.0) || !std::isfinite(k)) return fail(ctx, HS_EINVAL, "k must be positive and finite");
  for (int i = 0; i < S1 * S2; ++i)
    if (!std::isfinite(c[i])) return fail(ctx, HS_EINVAL, "non-finite sine coefficient");
  ctx->built = false;
  cudaStream_t s = ctx->stream;
  CK(cudaMemcpyAsync(ctx->d_c, c, sizeof(double) * S1 * S2, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(ctx->d_info, 0, sizeof(int) * ctx->ninfo, s));
  sine_eval_grid(s, ctx->d_c, S1, S2, ctx->d_xg, ctx->nL, ctx->d_sx16, ctx->d_sy16, ctx->d_T, ctx->d_Qg, ctx->d_q,
                 ctx->d_info + ctx->ninfo - 1);
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, ctx->d_info + ctx->ninfo - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (bad) return fail(ctx, HS_EINVAL, "1 - q <= 0 (or NaN) at a leaf node");
  return factor(ctx, k);
}

int hs_build_nodes(hs_ctx* ctx, const double* q_nodes, double k) {
  CKR(check_ctx(ctx, false));
  LaunchScope ls(ctx);
  if (!q_nodes) return fail(ctx, HS_EINVAL, "q_nodes is NULL");
  if (!(k > 0.0) || !std::isfinite(k)) return fail(ctx, HS_EINVAL, "k must be positive and finite");
  ctx->built = false;
  cudaStream_t s = ctx->stream;
  const long long n = (long long)ctx->nleaf * 256;
  CK(cudaMemcpyAsync(ctx->d_q, q_nodes, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(ctx->d_info, 0, sizeof(int) * ctx->ninfo, s));
  check_q(s, ctx->d_q, n, ctx->d_info + ctx->ninfo - 1);
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, ctx->d_info + ctx->ninfo - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (bad) return fail(ctx, HS_EINVAL, "1 - q <= 0 (or NaN) at a leaf node");
  return factor(ctx, k);
}

int hs_solve_dev(hs_ctx* ctx, const double* alphas, int M, const double* thetas, int P, double* ufar, void* stream) {
  CKR(check_ctx(ctx, true));
  LaunchScope ls(ctx);
  CKR(valid_angles(ctx, M, P));
  if (!alphas || !thetas || !ufar) return fail(ctx, HS_EINVAL, "NULL pointer");
  return solve_into(ctx, pick(ctx, stream), alphas, M, thetas, P, reinterpret_cast<double2*>(ufar));
}

int hs_solve(hs_ctx* ctx, const double* alphas, int M, const double* thetas, int P, double* ufar) {
  CKR(check_ctx(ctx, true));
  LaunchScope ls(ctx);
  CKR(valid_angles(ctx, M, P));
  if (!alphas || !thetas || !ufar) return fail(ctx, HS_EINVAL, "NULL pointer");
  cudaStream_t s = ctx->stream;
  double *da = nullptr, *dt = nullptr;
  double2* du = nullptr;
  CK(cudaMallocAsync(&da, sizeof(double) * M, s));
  CK(cudaMallocAsync(&dt, sizeof(double) * P, s));
  CK(cudaMallocAsync(&du, sizeof(double2) * M * P, s));
  CK(cudaMemcpyAsync(da, alphas, sizeof(double) * M, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dt, thetas, sizeof(double) * P, cudaMemcpyHostToDevice, s));
  int r = solve_into(ctx, s, da, M, dt, P, du);
  if (r == HS_OK) CK(cudaMemcpyAsync(ufar, du, sizeof(double2) * M * P, cudaMemcpyDeviceToHost, s));
  cudaFreeAsync(da, s);
  cudaFreeAsync(dt, s);
  cudaFreeAsync(du, s);
  CK(cudaStreamSynchronize(s));
  return r;
}

int hs_fields_dev(hs_ctx* ctx, const double* alphas, int M, double* u, void* stream) {
  CKR(check_ctx(ctx, true));
  LaunchScope ls(ctx);
  if (M <= 0 || M > 65535 || !alphas || !u) return fail(ctx, HS_EINVAL, "bad arguments");
  cudaStream_t s = pick(ctx, stream);
  const int nb = ctx->B.nb;
  Arena a;
  if (ctx->cfg.precision == HS_MIXED) {
    // refined FP64 fields; the far field is computed for one receiver (unused)
    CKR(ensure_ws(ctx, mixed_bytes(ctx, M, 1) + Arena::bytes((size_t)ctx->nleaf * NL * M, 16) + 4096, a));
    double2* X = a.get<double2>((size_t)ctx->nleaf * NL * M);
    double* th = a.get<double>(1);
    CK(cudaMemsetAsync(th, 0, sizeof(double), s));
    CKR(mixed_solve(ctx, s, alphas, M, th, 1, nullptr, X, a));
    leaf_to_nodes(s, X, ctx->nL, M, reinterpret_cast<double2*>(u));
    CK(cudaGetLastError());
    return HS_OK;
  }
  size_t need = 4 * Arena::bytes((size_t)nb * M, 16) + 2 * Arena::bytes(field_buf_elems(ctx, M), 16) +
                Arena::bytes(t3_elems(ctx, M), 16) + Arena::bytes((size_t)ctx->nleaf * NL * M, 16);
  CKR(ensure_ws(ctx, need, a));
  double2 *ui = a.get<double2>((size_t)nb * M), *dni = a.get<double2>((size_t)nb * M);
  double2 *f = a.get<double2>((size_t)nb * M), *g = a.get<double2>((size_t)nb * M);
  double2 *bufA = a.get<double2>(field_buf_elems(ctx, M)), *bufB = a.get<double2>(field_buf_elems(ctx, M));
  double2* T3 = a.get<double2>(t3_elems(ctx, M));
  double2* Uleaf = a.get<double2>((size_t)ctx->nleaf * NL * M);
  if (a.over) return fail(ctx, HS_ENOMEM, "workspace request beyond its sizing");
  CKR(root_solve(ctx, s, alphas, M, ui, dni, f, g));
  CKR(sweep_down(ctx, s, f, M, bufA, bufB, T3, Uleaf));
  leaf_to_nodes(s, Uleaf, ctx->nL, M, reinterpret_cast<double2*>(u));
  CK(cudaGetLastError());
  return HS_OK;
}

int hs_forward_dev(hs_ctx* ctx, const double* alphas, int M, const double* thetas, int P, double* ufar, double* u,
                   void* stream) {
  CKR(check_ctx(ctx, true));
  LaunchScope ls(ctx);
  CKR(valid_angles(ctx, M, P));
  if (!alphas || !thetas || !ufar || !u) return fail(ctx, HS_EINVAL, "NULL pointer");
  cudaStream_t s = pick(ctx, stream);
  const int nb = ctx->B.nb;
  Arena a;
  if (ctx->cfg.precision == HS_MIXED) {
    CKR(ensure_ws(ctx, mixed_bytes(ctx, M, P) + Arena::bytes((size_t)ctx->nleaf * NL * M, 16), a));
    double2* X = a.get<double2>((size_t)ctx->nleaf * NL * M);
    CKR(mixed_solve(ctx, s, alphas, M, thetas, P, reinterpret_cast<double2*>(ufar), X, a));
    leaf_to_nodes(s, X, ctx->nL, M, reinterpret_cast<double2*>(u));
    CK(cudaGetLastError());
    return HS_OK;
  }
  size_t need = 4 * Arena::bytes((size_t)nb * M, 16) + Arena::bytes((size_t)2 * nb * M, 16) +
                Arena::bytes((size_t)P * 2 * nb, 16) + 2 * Arena::bytes(field_buf_elems(ctx, M), 16) +
                Arena::bytes(t3_elems(ctx, M), 16) + Arena::bytes((size_t)ctx->nleaf * NL * M, 16);
  CKR(ensure_ws(ctx, need, a));
  double2 *ui = a.get<double2>((size_t)nb * M), *dni = a.get<double2>((size_t)nb * M);
  double2 *f = a.get<double2>((size_t)nb * M), *g = a.get<double2>((size_t)nb * M);
  double2* PS = a.get<double2>((size_t)2 * nb * M);
  double2* A2 = a.get<double2>((size_t)P * 2 * nb);
  double2 *bufA = a.get<double2>(field_buf_elems(ctx, M)), *bufB = a.get<double2>(field_buf_elems(ctx, M));
  double2* T3 = a.get<double2>(t3_elems(ctx, M));
  double2* Uleaf = a.get<double2>((size_t)ctx->nleaf * NL * M);
  if (a.over) return fail(ctx, HS_ENOMEM, "workspace request beyond its sizing");
  CKR(root_solve(ctx, s, alphas, M, ui, dni, f, g));
  boundary_data(s, nb, M, ctx->k, f, g, ui, dni, PS);
  farfield_matrix(s, ctx->B, ctx->k, ctx->cfg.R, thetas, P, A2);
  gemm<double2, double2, double2>(s, OP_T, OP_T, M, P, 2 * nb, make_double2(1, 0), PS, M, 0, A2, 2 * nb, 0,
                                  make_double2(0, 0), reinterpret_cast<double2*>(ufar), P, 0, 1);
  CKR(sweep_down(ctx, s, f, M, bufA, bufB, T3, Uleaf));
  leaf_to_nodes(s, Uleaf, ctx->nL, M, reinterpret_cast<double2*>(u));
  CK(cudaGetLastError());
  return HS_OK;
}

int hs_jacobian_dev(hs_ctx* ctx, const double* alphas, int M, const double* thetas, int P, double* J, void* stream) {
  CKR(check_ctx(ctx, true));
  LaunchScope ls(ctx);
  CKR(valid_angles(ctx, M, P));
  if (!alphas || !thetas || !J) return fail(ctx, HS_EINVAL, "NULL pointer");
  Arena a;
  CKR(ensure_ws(ctx, jacobian_bytes(ctx, M, P), a));
  return jacobian_into(ctx, pick(ctx, stream), alphas, M, thetas, P, reinterpret_cast<double2*>(J), a);
}

int hs_jacobian(hs_ctx* ctx, const double* alphas, int M, const double* thetas, int P, double* J) {
  CKR(check_ctx(ctx, true));
  LaunchScope ls(ctx);
  CKR(valid_angles(ctx, M, P));
  if (!alphas || !thetas || !J) return fail(ctx, HS_EINVAL, "NULL pointer");
  cudaStream_t s = ctx->stream;
  const size_t nJ = (size_t)M * P * ctx->S1 * ctx->S2;
  Arena a;
  size_t need = Arena::bytes(M, 8) + Arena::bytes(P, 8) + Arena::bytes(nJ, 16) + jacobian_bytes(ctx, M, P);
  CKR(ensure_ws(ctx, need, a));
  double* da = a.get<double>(M);
  double* dt = a.get<double>(P);
  double2* dJ = a.get<double2>(nJ);
  if (a.over) return fail(ctx, HS_ENOMEM, "workspace request beyond its sizing");
  CK(cudaMemcpyAsync(da, alphas, sizeof(double) * M, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dt, thetas, sizeof(double) * P, cudaMemcpyHostToDevice, s));
  CKR(jacobian_into(ctx, s, da, M, dt, P, dJ, a));
  CK(cudaMemcpyAsync(J, dJ, sizeof(double2) * nJ, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return HS_OK;
}

int hs_gn_step(hs_ctx* ctx, const double* data, const double* alphas, int M, const double* thetas, int P,
               double lambda_rel, double* c_inout, double* resid_norm_out) {
  CKR(check_ctx(ctx, true));
  LaunchScope ls(ctx);
  CKR(valid_angles(ctx, M, P));
  if (!data || !alphas || !thetas || !c_inout) return fail(ctx, HS_EINVAL, "NULL pointer");
  if (!(lambda_rel >= 0.0) || !std::isfinite(lambda_rel)) return fail(ctx, HS_EINVAL, "lambda_rel must be >= 0");
  const bool mixed = ctx->cfg.precision == HS_MIXED;
  cudaStream_t s = ctx->stream;
  const int MP = M * P, nm = ctx->S1 * ctx->S2;
  Arena a;
  size_t need = Arena::bytes(M, 8) + Arena::bytes(P, 8) + Arena::bytes((size_t)2 * MP, 8) +
                Arena::bytes(MP, 16) * 2 + Arena::bytes((size_t)2 * MP, 8) + Arena::bytes(8, 8) +
                Arena::bytes((size_t)MP * nm, 16) + Arena::bytes((size_t)2 * MP * nm, 8) +
                Arena::bytes((size_t)nm * nm, 8) + Arena::bytes(nm, 8) + Arena::bytes(nm, 4) +
                (g_oz_enabled ? Arena::bytes(normal_matrix_emulated_bytes(2 * MP, nm), 1) : 0) +
                std::max(jacobian_bytes(ctx, M, P),
                         4 * Arena::bytes((size_t)ctx->B.nb * M, 16) + Arena::bytes((size_t)2 * ctx->B.nb * M, 16) +
                             Arena::bytes((size_t)P * 2 * ctx->B.nb, 16));
  CKR(ensure_ws(ctx, need, a));
  double* da = a.get<double>(M);
  double* dt = a.get<double>(P);
  double* ddata = a.get<double>((size_t)2 * MP);
  double2* F = a.get<double2>(MP);
  double2* res = a.get<double2>(MP);
  double* rst = a.get<double>((size_t)2 * MP);
  double* nrm2 = a.get<double>(8);
  double2* J = a.get<double2>((size_t)MP * nm);
  double* Jst = a.get<double>((size_t)2 * MP * nm);
  double* A = a.get<double>((size_t)nm * nm);
  double* bv = a.get<double>(nm);
  int* piv = a.get<int>(nm);
  const size_t ozb = g_oz_enabled ? normal_matrix_emulated_bytes(2 * MP, nm) : 0;
  char* oz = ozb ? a.get<char>(ozb) : nullptr;
  if (a.over) return fail(ctx, HS_ENOMEM, "workspace request beyond its sizing");
  CK(cudaMemcpyAsync(da, alphas, sizeof(double) * M, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dt, thetas, sizeof(double) * P, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ddata, data, sizeof(double) * 2 * MP, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(nrm2, 0, sizeof(double), s));
  if (mixed) {  // refined far field, forward and adjoint fields from one call
    CKR(jacobian_into_mixed(ctx, s, da, M, dt, P, J, a, F));
    residual(s, ddata, F, MP, res, rst, nrm2);
  } else {
    Arena sub = a;  // the forward solve's scratch is reused by the Jacobian afterwards
    const int nb = ctx->B.nb;
    double2 *ui = sub.get<double2>((size_t)nb * M), *dni = sub.get<double2>((size_t)nb * M);
    double2 *f = sub.get<double2>((size_t)nb * M), *g = sub.get<double2>((size_t)nb * M);
    double2* PS = sub.get<double2>((size_t)2 * nb * M);
    double2* A2 = sub.get<double2>((size_t)P * 2 * nb);
    CKR(root_solve(ctx, s, da, M, ui, dni, f, g));
    boundary_data(s, nb, M, ctx->k, f, g, ui, dni, PS);
    farfield_matrix(s, ctx->B, ctx->k, ctx->cfg.R, dt, P, A2);
    gemm<double2, double2, double2>(s, OP_T, OP_T, M, P, 2 * nb, make_double2(1, 0), PS, M, 0, A2, 2 * nb, 0,
                                    make_double2(0, 0), F, P, 0, 1);
    residual(s, ddata, F, MP, res, rst, nrm2);
    CKR(jacobian_into(ctx, s, da, M, dt, P, J, a));
  }
  // normal equations in the real coefficients: A = Jst^T Jst, b = Jst^T rst (with the
  // emulated FP64 product the stack is formed transposed, Jst^T, its natural operand)
  bool emulated = false;
  if (oz) {
    split_stack_t(s, J, MP, nm, Jst);
    emulated = normal_matrix_emulated(s, Jst, 2 * MP, nm, A, oz, ozb);
    if (emulated)
      gemm<double, double, double>(s, OP_N, OP_N, nm, 1, 2 * MP, 1.0, Jst, 2 * MP, 0, rst, 1, 0, 0.0, bv, 1, 0, 1);
  }
  if (!emulated) {
    split_stack(s, J, MP, nm, Jst);
    normal_matrix(s, Jst, 2 * MP, nm, A);
    gemm<double, double, double>(s, OP_T, OP_N, nm, 1, 2 * MP, 1.0, Jst, nm, 0, rst, 1, 0, 0.0, bv, 1, 0, 1);
  }
  add_lambda(s, A, nm, lambda_rel);
  CK(cudaMemsetAsync(ctx->d_info, 0, sizeof(int) * ctx->ninfo, s));
  lu_factor<double>(s, A, nm, 0, nm, piv, 0, ctx->d_info, 1);
  lu_solve<double>(s, OP_N, A, nm, 0, nm, piv, 0, bv, 1, 0, 1, 1);
  std::vector<double> dc(nm);
  double r2 = 0.0;
  CK(cudaMemcpyAsync(dc.data(), bv, sizeof(double) * nm, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&r2, nrm2, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaGetLastError());
  CKR(check_info(ctx));
  for (int i = 0; i < nm; ++i) c_inout[i] += dc[i];
  if (resid_norm_out) *resid_norm_out = std::sqrt(r2);
  return HS_OK;
}

int hs_gn_step_lsqr(hs_ctx* ctx, const double* data, const double* alphas, int M, const double* thetas, int P,
                    const unsigned char* mask, double damp, double tol, int max_iter, int products,
                    double* c_inout, double* resid_norm_out, int* iters_out) {
  CKR(check_ctx(ctx, true));
  LaunchScope ls(ctx);
  CKR(valid_angles(ctx, M, P));
  const bool mixed = ctx->cfg.precision == HS_MIXED;
  if (!data || !alphas || !thetas || !c_inout) return fail(ctx, HS_EINVAL, "NULL pointer");
  if (!(damp >= 0.0) || !std::isfinite(damp) || !(tol >= 0.0) || max_iter < 1)
    return fail(ctx, HS_EINVAL, "damp and tol must be >= 0 and max_iter >= 1");
  if (products != HS_FP64 && products != HS_MIXED) return fail(ctx, HS_EINVAL, "products must be HS_FP64 or HS_MIXED");
  const bool p32 = products == HS_MIXED;
  // FP64 products with the emulated FP64 contraction: J formed once in FP64 and
  // read twice per iteration (exact transposes of one matrix); without the
  // emulation, J and J^H are applied from the fields by FP64 grid contractions
  const bool p64x = !p32 && g_oz_enabled;
  const int C32 = contract_chunk32(M, P, ctx->n14, ctx->S1, g_contract_budget);
  const int C64 = contract_chunk(M, P, ctx->n14, ctx->S1, g_contract_budget);
  cudaStream_t s = ctx->stream;
  const int MP = M * P, nm = ctx->S1 * ctx->S2, nX = ctx->n14, S1 = ctx->S1, S2 = ctx->S2;
  const size_t N = (size_t)nX * nX;
  const double k2 = ctx->k * ctx->k;
  const int nb = ctx->B.nb;
  // device buffers: inputs, residual, fields; then (reusing the solves' scratch)
  // the buffers of the two products
  const size_t far = 4 * Arena::bytes((size_t)nb * M, 16) + Arena::bytes((size_t)2 * nb * M, 16) +
                     Arena::bytes((size_t)P * 2 * nb, 16);
  // the FP64 products' buffers (G1, qv, h, Y, fc, T1) or the FP32 Jacobian's
  const size_t prod = Arena::bytes(nm, 8) * 2 + Arena::bytes(MP, 16) +
                      (p32 ? Arena::bytes((size_t)MP * nm, 8) + Arena::bytes((size_t)nX * S1, 8) +
                                 Arena::bytes((size_t)nX * S2, 4) + Arena::bytes(N * C32, 8) +
                                 Arena::bytes((size_t)nX * S1 * C32, 8) +
                                 Arena::bytes((size_t)gemvT_parts(MP) * nm, 8)
                       : p64x ? Arena::bytes((size_t)MP * nm, 16) + Arena::bytes(N * C64, 16) +
                                    Arena::bytes((size_t)nX * S1 * C64, 16) +
                                    Arena::bytes(contract_emulated_bytes(C64, nX, S1, S2), 1) +
                                    Arena::bytes((size_t)gemvT_parts(MP) * nm, 8)
                              : Arena::bytes((size_t)S2 * nX, 8) + Arena::bytes(N, 8) * 2 + Arena::bytes(N * M, 16) +
                                    Arena::bytes(MP, 16) + Arena::bytes((size_t)S1 * nX, 8));
  const size_t need = Arena::bytes(M, 8) + Arena::bytes(P, 8) + Arena::bytes((size_t)2 * MP, 8) +
                      Arena::bytes(8, 8) + Arena::bytes(MP, 16) * 2 + Arena::bytes(N * M, 16) +
                      Arena::bytes(N * P, 16) +
                      std::max({far, mixed ? mixed_fields_bytes(ctx, M, P) : fields_and_adjoint_bytes(ctx, M, P), prod});
  Arena a;
  CKR(ensure_ws(ctx, need, a));
  double* da = a.get<double>(M);
  double* dt = a.get<double>(P);
  double* ddata = a.get<double>((size_t)2 * MP);
  double* nrm2 = a.get<double>(8);
  double2* F = a.get<double2>(MP);
  double2* res = a.get<double2>(MP);
  double2* Ug = a.get<double2>(N * M);
  double2* Zg = a.get<double2>(N * P);
  if (a.over) return fail(ctx, HS_ENOMEM, "workspace request beyond its sizing");
  CK(cudaMemcpyAsync(da, alphas, sizeof(double) * M, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dt, thetas, sizeof(double) * P, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ddata, data, sizeof(double) * 2 * MP, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(nrm2, 0, sizeof(double), s));
  if (mixed) {  // refined far field and forward fields; the adjoint refined to the tolerance, or,
                // for the FP32 Jacobian, with one FP64-residual correction (its error is then
                // below that matrix's own FP32 rounding)
    Arena sub = a;
    CKR(mixed_fields_and_adjoint(ctx, s, da, M, dt, P, F, Ug, Zg, sub, p32 ? 2 : 0));
  } else {  // forward far field F(c)
    Arena sub = a;
    double2 *ui = sub.get<double2>((size_t)nb * M), *dni = sub.get<double2>((size_t)nb * M);
    double2 *f = sub.get<double2>((size_t)nb * M), *g = sub.get<double2>((size_t)nb * M);
    double2* PS = sub.get<double2>((size_t)2 * nb * M);
    double2* A2 = sub.get<double2>((size_t)P * 2 * nb);
    if (sub.over) return fail(ctx, HS_ENOMEM, "workspace request beyond its sizing");
    CKR(root_solve(ctx, s, da, M, ui, dni, f, g));
    boundary_data(s, nb, M, ctx->k, f, g, ui, dni, PS);
    farfield_matrix(s, ctx->B, ctx->k, ctx->cfg.R, dt, P, A2);
    gemm<double2, double2, double2>(s, OP_T, OP_T, M, P, 2 * nb, make_double2(1, 0), PS, M, 0, A2, 2 * nb, 0,
                                    make_double2(0, 0), F, P, 0, 1);
  }
  residual(s, ddata, F, MP, res, nullptr, nrm2);  // r = data - F
  if (!mixed) {
    Arena sub = a;
    CKR(fields_and_adjoint(ctx, s, da, M, dt, P, Ug, Zg, sub));
  }
  interior_sine_tables(s, ctx->d_xint, nX, S1, S2, ctx->d_sxi, ctx->d_syi);
  double* dv = a.get<double>(nm);
  double* dg = a.get<double>(nm);
  double2* dy = a.get<double2>(MP);
  double *G1 = nullptr, *qv = nullptr, *h = nullptr, *T1 = nullptr;
  double2 *Y = nullptr, *fc = nullptr;
  float2 *J32 = nullptr, *sxc = nullptr, *W32 = nullptr, *T32 = nullptr;
  float* sy32 = nullptr;
  double* partT = nullptr;
  double2 *J64 = nullptr, *W64 = nullptr, *T64 = nullptr;
  char* oz = nullptr;
  const size_t ozb = p64x ? contract_emulated_bytes(C64, nX, S1, S2) : 0;
  if (p64x) {
    J64 = a.get<double2>((size_t)MP * nm);
    W64 = a.get<double2>(N * C64);
    T64 = a.get<double2>((size_t)nX * S1 * C64);
    oz = a.get<char>(ozb);
    partT = a.get<double>((size_t)gemvT_parts(MP) * nm);
  } else if (!p32) {
    G1 = a.get<double>((size_t)S2 * nX);
    qv = a.get<double>(N);
    h = a.get<double>(N);
    Y = a.get<double2>(N * M);
    fc = a.get<double2>(MP);
    T1 = a.get<double>((size_t)S1 * nX);
  } else {
    J32 = a.get<float2>((size_t)MP * nm);
    sxc = a.get<float2>((size_t)nX * S1);
    sy32 = a.get<float>((size_t)nX * S2);
    W32 = a.get<float2>(N * C32);
    T32 = a.get<float2>((size_t)nX * S1 * C32);
    partT = a.get<double>((size_t)gemvT_parts(MP) * nm);
  }
  if (a.over) return fail(ctx, HS_ENOMEM, "workspace request beyond its sizing");
  if (p32) {
    Phase phj("hs_jacobian32");
    contract_jacobian32(s, Ug, Zg, M, P, nX, ctx->d_sxi, ctx->d_syi, S1, S2, k2, J32, sxc, sy32, W32, T32, C32);
  }
  if (p64x) {
    Phase phj("hs_jacobian_contract");
    contract_jacobian(s, Ug, Zg, M, P, nX, ctx->d_sxi, ctx->d_syi, S1, S2, k2, J64, W64, T64, C64, oz, ozb);
  }
  std::vector<unsigned char> keep(nm, 1);
  if (mask)
    for (int i = 0; i < nm; ++i) keep[i] = mask[i] ? 1 : 0;
  // A = [Re J; Im J] restricted to the kept columns, as products on the GPU
  std::vector<double2> hy(MP);
  auto matvec = [&](const std::vector<double>& v, std::vector<double>& out) {  // out (2 MP) = A v
    CK(cudaMemcpyAsync(dv, v.data(), sizeof(double) * nm, cudaMemcpyHostToDevice, s));
    if (p32)
      gemv32(s, J32, MP, nm, dv, dy);
    else if (p64x)
      gemv64(s, J64, MP, nm, dv, dy);
    else
      apply_J(s, Ug, Zg, M, P, nX, ctx->d_sxi, ctx->d_syi, S1, S2, k2, dv, G1, qv, Y, dy);
    CK(cudaMemcpyAsync(hy.data(), dy, sizeof(double2) * MP, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int i = 0; i < MP; ++i) {
      out[i] = hy[i].x;
      out[MP + i] = hy[i].y;
    }
    return HS_OK;
  };
  auto rmatvec = [&](const std::vector<double>& u, std::vector<double>& out) {  // out (nm) = A^T u
    for (int i = 0; i < MP; ++i) hy[i] = make_double2(u[i], u[MP + i]);
    CK(cudaMemcpyAsync(dy, hy.data(), sizeof(double2) * MP, cudaMemcpyHostToDevice, s));
    if (p32)
      gemvT32(s, J32, MP, nm, dy, partT, dg);
    else if (p64x)
      gemvT64(s, J64, MP, nm, dy, partT, dg);
    else
      apply_JH(s, Ug, Zg, M, P, nX, ctx->d_sxi, ctx->d_syi, S1, S2, k2, dy, fc, Y, h, T1, dg);
    CK(cudaMemcpyAsync(out.data(), dg, sizeof(double) * nm, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int i = 0; i < nm; ++i)
      if (!keep[i]) out[i] = 0.0;
    return HS_OK;
  };
  auto norm = [](const std::vector<double>& z) {
    double acc = 0.0;
    for (double e : z) acc += e * e;
    return std::sqrt(acc);
  };
  // LSQR (Paige and Saunders): Golub-Kahan bidiagonalisation started from
  // b = [Re r; Im r], plane rotations (first the damping term, then beta)
  std::vector<double> b(2 * (size_t)MP), u(2 * (size_t)MP), t2(2 * (size_t)MP);
  std::vector<double> x(nm, 0.0), v(nm), w(nm), tn(nm);
  {
    std::vector<double2> hr(MP);
    CK(cudaMemcpyAsync(hr.data(), res, sizeof(double2) * MP, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int i = 0; i < MP; ++i) {
      b[i] = hr[i].x;
      b[MP + i] = hr[i].y;
    }
  }
  Phase ph("hs_gn_lsqr");
  int it = 0;
  double beta = norm(b);
  if (beta > 0.0) {
    for (size_t i = 0; i < b.size(); ++i) u[i] = b[i] / beta;
    CKR(rmatvec(u, v));
    double alpha = norm(v);
    if (alpha > 0.0) {
      for (double& e : v) e /= alpha;
      w = v;
      double phibar = beta, rhobar = alpha, anorm2 = 0.0, res2 = 0.0;
      const double beta1 = beta;
      while (it < max_iter) {
        ++it;
        CKR(matvec(v, t2));
        for (size_t i = 0; i < u.size(); ++i) u[i] = t2[i] - alpha * u[i];
        beta = norm(u);
        if (beta > 0.0)
          for (double& e : u) e /= beta;
        anorm2 += alpha * alpha + beta * beta + damp * damp;
        CKR(rmatvec(u, tn));
        for (int i = 0; i < nm; ++i) v[i] = tn[i] - beta * v[i];
        alpha = norm(v);
        if (alpha > 0.0)
          for (double& e : v) e /= alpha;
        const double rhobar1 = std::hypot(rhobar, damp);
        const double c1 = rhobar / rhobar1, s1 = damp / rhobar1;
        const double psi = s1 * phibar;
        phibar = c1 * phibar;
        const double rho = std::hypot(rhobar1, beta);
        const double c = rhobar1 / rho, sn = beta / rho;
        const double theta = sn * alpha;
        rhobar = -c * alpha;
        const double phi = c * phibar;
        phibar = sn * phibar;
        for (int i = 0; i < nm; ++i) {
          x[i] += (phi / rho) * w[i];
          w[i] = v[i] - (theta / rho) * w[i];
        }
        res2 += psi * psi;
        const double rnorm = std::sqrt(phibar * phibar + res2);
        const double arnorm = alpha * std::fabs(c) * std::fabs(phibar);
        const double test1 = rnorm / beta1;
        const double test2 = rnorm > 0.0 ? arnorm / (std::sqrt(anorm2) * rnorm) : 0.0;
        if (test1 <= tol || test2 <= tol || alpha == 0.0 || beta == 0.0) break;
      }
    }
  }
  double r2 = 0.0;
  CK(cudaMemcpyAsync(&r2, nrm2, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  if ((p32 || p64x) && tc_timed_out(s)) return fail(ctx, HS_ETIMEOUT, "a tensor-core GEMM wait gave up");
  for (int i = 0; i < nm; ++i) c_inout[i] += x[i];
  if (resid_norm_out) *resid_norm_out = std::sqrt(r2);
  if (iters_out) *iters_out = it;
  return HS_OK;
}

int hs_gradient_dev(hs_ctx* ctx, const double* data, const double* alphas, int M, const double* thetas, int P,
                    double* grad, double* misfit_out, void* stream) {
  CKR(check_ctx(ctx, true));
  LaunchScope ls(ctx);
  CKR(valid_angles(ctx, M, P));
  if (!data || !alphas || !thetas || !grad || !misfit_out) return fail(ctx, HS_EINVAL, "NULL pointer");
  Arena a;
  CKR(ensure_ws(ctx, gradient_bytes(ctx, M, P), a));
  return gradient_core(ctx, pick(ctx, stream), data, alphas, M, thetas, P, grad, misfit_out, a);
}

int hs_gradient(hs_ctx* ctx, const double* data, const double* alphas, int M, const double* thetas, int P,
                double* grad, double* misfit_out) {
  CKR(check_ctx(ctx, true));
  LaunchScope ls(ctx);
  CKR(valid_angles(ctx, M, P));
  if (!data || !alphas || !thetas || !grad) return fail(ctx, HS_EINVAL, "NULL pointer");
  cudaStream_t s = ctx->stream;
  const int MP = M * P, nm = ctx->S1 * ctx->S2;
  Arena a;
  size_t need = Arena::bytes(M, 8) + Arena::bytes(P, 8) + Arena::bytes((size_t)2 * MP, 8) + Arena::bytes(nm, 8) +
                Arena::bytes(8, 8) + gradient_bytes(ctx, M, P);
  CKR(ensure_ws(ctx, need, a));
  double* da = a.get<double>(M);
  double* dt = a.get<double>(P);
  double* ddata = a.get<double>((size_t)2 * MP);
  double* dg = a.get<double>(nm);
  double* dm = a.get<double>(8);
  if (a.over) return fail(ctx, HS_ENOMEM, "workspace request beyond its sizing");
  CK(cudaMemcpyAsync(da, alphas, sizeof(double) * M, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dt, thetas, sizeof(double) * P, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ddata, data, sizeof(double) * 2 * MP, cudaMemcpyHostToDevice, s));
  CKR(gradient_core(ctx, s, ddata, da, M, dt, P, dg, dm, a));
  double mis = 0.0;
  CK(cudaMemcpyAsync(grad, dg, sizeof(double) * nm, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&mis, dm, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (misfit_out) *misfit_out = mis;
  return HS_OK;
}

long long hs_launch_count(const hs_ctx* ctx) { return ctx ? ctx->launches : 0; }

int hs_refine_stats(const hs_ctx* ctx, int* iterations, double* last_update, double* est_error) {
  if (!ctx) return HS_EINVAL;
  if (iterations) *iterations = ctx->refine_iters;
  if (last_update) *last_update = ctx->refine_update;
  if (est_error) *est_error = ctx->refine_est;
  return HS_OK;
}

int hs_build_phase_ms(const hs_ctx* ctx, double* interior_ms, double* boundary_ms) {
  if (!ctx) return HS_EINVAL;
  if (interior_ms) *interior_ms = ctx->t_interior;
  if (boundary_ms) *boundary_ms = ctx->t_bdry;
  return HS_OK;
}

int hs_adjoint_refine_stats(const hs_ctx* ctx, int* iterations, double* last_update, double* est_error) {
  if (!ctx) return HS_EINVAL;
  if (iterations) *iterations = ctx->adj_iters;
  if (last_update) *last_update = ctx->adj_update;
  if (est_error) *est_error = ctx->adj_est;
  return HS_OK;
}

const char* hs_last_error(const hs_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

void hs_destroy(hs_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->cfg.device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  ctx->fgraph.reset();
  ctx->pgraph[0].reset();
  ctx->pgraph[1].reset();
  for (auto& e : ctx->ph_ev)
    if (e) cudaEventDestroy(e);
  for (void* p : ctx->allocs) cudaFree(p);
  if (ctx->ws_base) cudaFree(ctx->ws_base);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

}  // extern "C"
