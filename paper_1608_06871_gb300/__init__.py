"""Python binding of libhs (include/hs.h): argument marshalling only.

Every numerical step runs in the CUDA library; this module converts NumPy
arrays (host calls) or torch CUDA tensors (``*_dev`` calls) to pointers and
raises ``HSError`` on a non-zero status.  There is no CPU fallback: if
``libhs.so`` has not been built, or no GPU is present, the calls fail.

The names mirror the C ABI: ``hs_create``, ``hs_build``, ``hs_build_nodes``,
``hs_node_coords``, ``hs_solve``, ``hs_solve_dev``, ``hs_fields_dev``,
``hs_jacobian``, ``hs_jacobian_dev``, ``hs_gn_step``, ``hs_gradient``,
``hs_gradient_dev``, ``hs_launch_count``, ``hs_last_error``, ``hs_destroy``.
A small ``Solver`` class wraps a context.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhs.so")

HS_OK, HS_EINVAL, HS_ENOTBUILT, HS_ENOMEM, HS_ECUDA, HS_ESINGULAR, HS_ENOCONV, HS_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7
HS_FP64, HS_MIXED = 0, 1
_NAMES = {0: "HS_OK", -1: "HS_EINVAL", -2: "HS_ENOTBUILT", -3: "HS_ENOMEM", -4: "HS_ECUDA",
          -5: "HS_ESINGULAR", -6: "HS_ENOCONV", -7: "HS_ETIMEOUT"}


class HSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class hs_config(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double), ("leaves_per_side", ctypes.c_int), ("S1", ctypes.c_int),
                ("S2", ctypes.c_int), ("precision", ctypes.c_int), ("device", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("refine_tol", ctypes.c_double), ("refine_max_iter", ctypes.c_int),
                ("bm_eta", ctypes.c_double), ("leaf_impedance", ctypes.c_int)]


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.c_int

_SIGS = {
    "hs_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(hs_config)]),
    "hs_build": (_I, [_P, _D, _I, _I, ctypes.c_double]),
    "hs_build_nodes": (_I, [_P, _D, ctypes.c_double]),
    "hs_node_coords": (_I, [_P, _D, _D]),
    "hs_solve": (_I, [_P, _D, _I, _D, _I, _D]),
    "hs_solve_dev": (_I, [_P, _P, _I, _P, _I, _P, _P]),
    "hs_fields_dev": (_I, [_P, _P, _I, _P, _P]),
    "hs_forward_dev": (_I, [_P, _P, _I, _P, _I, _P, _P, _P]),
    "hs_solve_noalloc": (_I, [_P, _P, _I, _P, _I, _P, _P]),
    "hs_jacobian": (_I, [_P, _D, _I, _D, _I, _D]),
    "hs_jacobian_dev": (_I, [_P, _P, _I, _P, _I, _P, _P]),
    "hs_gn_step": (_I, [_P, _D, _D, _I, _D, _I, ctypes.c_double, _D, _D]),
    "hs_gn_step_lsqr": (_I, [_P, _D, _D, _I, _D, _I, _P, ctypes.c_double, ctypes.c_double, _I, _I, _D, _D,
                             ctypes.POINTER(_I)]),
    "hs_gradient": (_I, [_P, _D, _D, _I, _D, _I, _D, _D]),
    "hs_gradient_dev": (_I, [_P, _P, _P, _I, _P, _I, _P, _P, _P]),
    "hs_launch_count": (ctypes.c_longlong, [_P]),
    "hs_last_error": (ctypes.c_char_p, [_P]),
    "hs_destroy": (None, [_P]),
    "hs_prof_start": (_I, [_I]),
    "hs_prof_stop": (_I, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_longlong)]),
    "hs_peak_fp64": (_I, [_I, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "hs_peak_fp32": (_I, [_I, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "hs_refine_stats": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double)]),
    "hs_adjoint_refine_stats": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]),
    "hs_build_phase_ms": (_I, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "hs_set_tensor_cores": (_I, [_I]),
    "hs_set_autotune": (_I, [_I]),
    "hs_set_tc_margin": (_I, [ctypes.c_double]),
    "hs_gemm32": (_I, [_I, _I, _I, _I, _P, _P, _P, _I, _I, _P, _P]),
    "hs_fail_next_allocs": (_I, [_I]),
    "hs_raise_tc_timeout": (_I, [_I]),
    "hs_set_graphs": (_I, [_I]),
    "hs_set_contract_budget": (_I, [ctypes.c_ulonglong]),
    "hs_cgemm32": (_I, [_I, _I, _I, _P, _P, _P, _I, _P, ctypes.POINTER(_I)]),
    "hs_lu_solve": (_I, [_I, _I, _I, _P, _P, _I, _P]),
    "hs_zgemm": (_I, [_I, _I, _I, _I, _I, _P, _P, _P, _I, _P]),
    "hs_dgemm_emulated": (_I, [_I, _I, _I, _P, _P, _P, _I, _P]),
    "hs_set_fp64_emulation": (_I, [_I]),
    "hs_jacobian32_products": (_I, [ctypes.c_longlong, _I, _P, _P, _P, _P, _P, _P]),
}


def lib() -> ctypes.CDLL:
    """Load libhs.so (built in-tree by ``paper_1608_06871_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1608_06871_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _check(ctx, code: int):
    if code != HS_OK:
        msg = lib().hs_last_error(ctx)
        raise HSError(code, msg.decode() if msg else "")


# ---- C-ABI mirrors ------------------------------------------------------------
def hs_create(leaves_per_side: int, S1: int, S2: int, R: float = 3.0, precision: int = HS_FP64, device: int = 0,
              stream: int | None = None, refine_tol: float = 0.0, refine_max_iter: int = 0, bm_eta: float = 0.0,
              leaf_impedance: bool = False):
    cfg = hs_config(R, leaves_per_side, S1, S2, precision, device, stream, refine_tol, refine_max_iter, bm_eta,
                    1 if leaf_impedance else 0)
    ctx = _P()
    code = lib().hs_create(ctypes.byref(ctx), ctypes.byref(cfg))
    if code != HS_OK:
        raise HSError(code, "hs_create failed")
    return ctx


def hs_build(ctx, c: np.ndarray, k: float):
    c = _f64(c)
    _check(ctx, lib().hs_build(ctx, _dp(c), c.shape[0], c.shape[1], float(k)))


def hs_build_nodes(ctx, q_nodes: np.ndarray, k: float):
    q = _f64(q_nodes)
    _check(ctx, lib().hs_build_nodes(ctx, _dp(q), float(k)))


def hs_node_coords(ctx, n_nodes: int):
    x = np.empty(n_nodes)
    y = np.empty(n_nodes)
    _check(ctx, lib().hs_node_coords(ctx, _dp(x), _dp(y)))
    return x, y


def hs_solve(ctx, alphas, thetas) -> np.ndarray:
    a, t = _f64(alphas), _f64(thetas)
    out = np.empty((len(a), len(t), 2))
    _check(ctx, lib().hs_solve(ctx, _dp(a), len(a), _dp(t), len(t), _dp(out)))
    return out[..., 0] + 1j * out[..., 1]


def _tp(t) -> int:
    return t.data_ptr()


def hs_solve_dev(ctx, alphas, thetas, ufar, stream: int | None = None):
    """alphas, thetas: float64 CUDA tensors; ufar: float64 CUDA tensor (M, P, 2)."""
    _check(ctx, lib().hs_solve_dev(ctx, _tp(alphas), alphas.numel(), _tp(thetas), thetas.numel(), _tp(ufar), stream))


def hs_solve_noalloc(ctx, alphas, thetas, ufar, stream: int | None = None):
    """As hs_solve_dev, but the library allocates nothing: its temporaries come from
    a fixed 16 MiB device array (for callers whose device memory belongs to another
    allocator).  Needs 16 * 56 n_L * (6 M + 2 P) bytes at most 16 MiB."""
    _check(ctx, lib().hs_solve_noalloc(ctx, _tp(alphas), alphas.numel(), _tp(thetas), thetas.numel(), _tp(ufar),
                                       stream))


def hs_forward_dev(ctx, alphas, thetas, ufar, u, stream: int | None = None):
    """Far field (M, P, 2) and total fields on every leaf node (M, n_L^2, 256, 2), float64 CUDA tensors."""
    _check(ctx, lib().hs_forward_dev(ctx, _tp(alphas), alphas.numel(), _tp(thetas), thetas.numel(), _tp(ufar),
                                     _tp(u), stream))


def hs_fields_dev(ctx, alphas, u, stream: int | None = None):
    """u: float64 CUDA tensor (M, n_L^2, 256, 2): total fields on the leaf nodes."""
    _check(ctx, lib().hs_fields_dev(ctx, _tp(alphas), alphas.numel(), _tp(u), stream))


def hs_jacobian(ctx, alphas, thetas, S1: int, S2: int) -> np.ndarray:
    a, t = _f64(alphas), _f64(thetas)
    out = np.empty((len(a) * len(t), S1 * S2, 2))
    _check(ctx, lib().hs_jacobian(ctx, _dp(a), len(a), _dp(t), len(t), _dp(out)))
    return out[..., 0] + 1j * out[..., 1]


def hs_jacobian_dev(ctx, alphas, thetas, J, stream: int | None = None):
    _check(ctx, lib().hs_jacobian_dev(ctx, _tp(alphas), alphas.numel(), _tp(thetas), thetas.numel(), _tp(J), stream))


def _cplx_pairs(z) -> np.ndarray:
    z = np.asarray(z, dtype=np.complex128)
    return np.ascontiguousarray(np.stack([z.real, z.imag], axis=-1))


def hs_gn_step(ctx, data, alphas, thetas, lambda_rel: float, c):
    """Returns (new coefficients, ||data - F(c)||) -- eq. normaleq."""
    d = _cplx_pairs(data)
    a, t = _f64(alphas), _f64(thetas)
    c2 = _f64(c).copy()
    rn = ctypes.c_double(0.0)
    _check(ctx, lib().hs_gn_step(ctx, _dp(d), _dp(a), len(a), _dp(t), len(t), float(lambda_rel), _dp(c2),
                                 ctypes.byref(rn)))
    return c2, rn.value


def hs_gn_step_lsqr(ctx, data, alphas, thetas, c, mask=None, damp: float = 0.0, tol: float = 1e-3,
                    max_iter: int = 100, products: int = HS_FP64):
    """Returns (new coefficients, ||data - F(c)||, LSQR iterations): the Gauss-Newton step with
    LSQR on the linearized problem (Sec. 4), dc restricted to mask (boolean, shape of c);
    products = HS_MIXED runs the grid contractions in FP32 on the tensor cores."""
    d = _cplx_pairs(data)
    a, t = _f64(alphas), _f64(thetas)
    c2 = _f64(c).copy()
    m = None if mask is None else np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).ravel())
    if m is not None and m.size != c2.size:
        raise ValueError("mask must have the shape of c")
    rn = ctypes.c_double(0.0)
    it = _I(0)
    _check(ctx, lib().hs_gn_step_lsqr(ctx, _dp(d), _dp(a), len(a), _dp(t), len(t),
                                      None if m is None else m.ctypes.data_as(_P), float(damp), float(tol),
                                      int(max_iter), int(products), _dp(c2), ctypes.byref(rn), ctypes.byref(it)))
    return c2, rn.value, it.value


def hs_gradient(ctx, data, alphas, thetas, S1: int, S2: int):
    """Returns (grad of 0.5 ||F(c) - data||^2 w.r.t. c as (S1, S2), misfit)."""
    d = _cplx_pairs(data)
    a, t = _f64(alphas), _f64(thetas)
    g = np.empty((S1, S2))
    mis = ctypes.c_double(0.0)
    _check(ctx, lib().hs_gradient(ctx, _dp(d), _dp(a), len(a), _dp(t), len(t), _dp(g), ctypes.byref(mis)))
    return g, mis.value


def hs_gradient_dev(ctx, data, alphas, thetas, grad, misfit, stream: int | None = None):
    _check(ctx, lib().hs_gradient_dev(ctx, _tp(data), _tp(alphas), alphas.numel(), _tp(thetas), thetas.numel(),
                                      _tp(grad), _tp(misfit), stream))


def hs_launch_count(ctx) -> int:
    return int(lib().hs_launch_count(ctx))


def hs_last_error(ctx) -> str:
    return lib().hs_last_error(ctx).decode()


def hs_destroy(ctx):
    lib().hs_destroy(ctx)


# ---- measurement hooks (include/hs_diag.h) --------------------------------------
HS_PROF_GEMM_FP64 = 1
HS_PROF_GEMM_FP32 = 2
HS_PROF_GEMM_TC = 3
HS_PROF_GEMM_EMU = 4


def hs_prof_start(family: int = HS_PROF_GEMM_FP64):
    _check(None, lib().hs_prof_start(family))


def hs_prof_stop():
    """Returns (total kernel ms, total algorithmic flops, launches) of the recorded family."""
    ms, fl, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
    _check(None, lib().hs_prof_stop(ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(n)))
    return ms.value, fl.value, n.value


def hs_refine_stats(ctx):
    """(refinement passes, last relative far-field change, estimated relative
    far-field error) of the last HS_MIXED solve."""
    it, up, est = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().hs_refine_stats(ctx, ctypes.byref(it), ctypes.byref(up), ctypes.byref(est)))
    return it.value, up.value, est.value


def hs_build_phase_ms(ctx):
    """(interior ms, exterior ms) of the last build: leaves + merges, then layer potentials +
    coupled root system; (-1, -1) after a build replayed from a CUDA graph."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().hs_build_phase_ms(ctx, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def hs_adjoint_refine_stats(ctx):
    """(passes, last relative change, estimated relative error) of the adjoint fields
    of the last HS_MIXED Jacobian, gradient or Gauss-Newton step."""
    it, up, est = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().hs_adjoint_refine_stats(ctx, ctypes.byref(it), ctypes.byref(up), ctypes.byref(est)))
    return it.value, up.value, est.value


def hs_peak_fp64(device: int = 0, ms: float = 300.0) -> float:
    t = ctypes.c_double()
    _check(None, lib().hs_peak_fp64(device, float(ms), ctypes.byref(t)))
    return t.value


def hs_peak_fp32(device: int = 0, ms: float = 300.0) -> float:
    t = ctypes.c_double()
    _check(None, lib().hs_peak_fp32(device, float(ms), ctypes.byref(t)))
    return t.value


def hs_set_graphs(enable: bool):
    _check(None, lib().hs_set_graphs(1 if enable else 0))


def hs_set_contract_budget(nbytes: int):
    """Scratch bytes per chunk of the Jacobian contraction (0 = the default 1 GiB)."""
    _check(None, lib().hs_set_contract_budget(int(nbytes)))


def hs_fail_next_allocs(n: int):
    """Test hook: the next n device allocations of the library fail with HS_ENOMEM (host side)."""
    _check(None, lib().hs_fail_next_allocs(int(n)))


def hs_raise_tc_timeout(device: int = 0):
    """Test hook: set the device's tensor-core timeout flag from the host; the next
    checking call reports HS_ETIMEOUT."""
    _check(None, lib().hs_raise_tc_timeout(int(device)))


def hs_set_tensor_cores(enable):
    """0 / False: SIMT FP32 products; 1 / True: per-shape choice (tensor cores where measured
    clearly faster); 2: tensor cores for every supported product."""
    _check(None, lib().hs_set_tensor_cores(int(enable)))


def hs_set_autotune(enable: bool):
    _check(None, lib().hs_set_autotune(1 if enable else 0))


def hs_set_tc_margin(margin: float):
    _check(None, lib().hs_set_tc_margin(float(margin)))


def hs_zgemm(A, B, C, transA: bool = False, transB: bool = False, accumulate: bool = False, stream: int = 0):
    """C = op(A) op(B) (+ C) for contiguous complex128 CUDA matrices (library FP64 GEMM)."""
    m = A.shape[1] if transA else A.shape[0]
    k = A.shape[0] if transA else A.shape[1]
    n = B.shape[0] if transB else B.shape[1]
    _check(None, lib().hs_zgemm(int(transA), int(transB), m, n, k, ctypes.c_void_p(A.data_ptr()),
                                ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(C.data_ptr()), int(accumulate),
                                ctypes.c_void_p(stream)))


def hs_dgemm_emulated(A, B, C, stream: int = 0):
    """C[b] = A[b] @ B[b] for contiguous float64 CUDA tensors of shape (batch, m, k), (batch, k, n),
    (batch, m, n) by the emulated FP64 product on the tensor cores (exact BF16 slices)."""
    batch, m, k = A.shape
    n = B.shape[2]
    _check(None, lib().hs_dgemm_emulated(m, n, k, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                         ctypes.c_void_p(C.data_ptr()), batch, ctypes.c_void_p(stream)))


def hs_set_fp64_emulation(enable: bool):
    _check(None, lib().hs_set_fp64_emulation(1 if enable else 0))


def hs_lu_solve(A, B, stream: int = 0):
    """Solve A[b] X[b] = B[b] in place in B (A overwritten by its LU factors) for
    contiguous complex128 (HS_FP64) or complex64 (HS_MIXED) CUDA tensors of
    shape (batch, n, n) and (batch, n, nrhs)."""
    batch, n, _ = A.shape
    prec = HS_FP64 if A.dtype == B.dtype and str(A.dtype) == "torch.complex128" else HS_MIXED
    _check(None, lib().hs_lu_solve(prec, n, B.shape[2], ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                   batch, ctypes.c_void_p(stream)))


def hs_cgemm32(A, B, out, stream: int = 0) -> bool:
    """out[b] = A[b] @ B[b] for contiguous complex64 CUDA tensors of shape
    (batch, m, k), (batch, k, n), (batch, m, n).  Returns True when the
    tensor-core kernel ran."""
    batch, m, k = A.shape
    n = B.shape[2]
    used = ctypes.c_int()
    _check(None, lib().hs_cgemm32(m, n, k, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), batch, ctypes.c_void_p(stream),
                                  ctypes.byref(used)))
    return bool(used.value)


def hs_gemm32(A, B, out, b_shared: bool = False, stream: int = 0) -> bool:
    """out[b] = A[b] @ B[b] (B[0] for every b when b_shared) for contiguous CUDA tensors:
    complex64 A, B, out (mode 2), float32 A with complex64 B and out (mode 1), or float32
    A, B, out (mode 0).  Returns True when the tensor cores ran it."""
    batch, m, k = A.shape
    n = B.shape[2]
    mode = 2 if A.is_complex() else (1 if B.is_complex() else 0)
    used = ctypes.c_int()
    _check(None, lib().hs_gemm32(mode, m, n, k, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), batch, 1 if b_shared else 0,
                                 ctypes.c_void_p(stream), ctypes.byref(used)))
    return bool(used.value)


def hs_jacobian32_products(J, v, y, u, g, stream: int = 0):
    """y = J @ v and g = Re(J^H u) for a contiguous complex64 CUDA matrix J (rows, n), float64 v (n),
    complex128 y and u (rows) and float64 g (n): the products LSQR applies to the FP32 Jacobian."""
    rows, n = J.shape
    _check(None, lib().hs_jacobian32_products(rows, n, ctypes.c_void_p(J.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                              ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                              ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(stream)))


class Solver:
    """One factorisation context: hs_create + hs_build, with NumPy host calls."""

    def __init__(self, leaves_per_side: int, S1: int, S2: int, R: float = 3.0, precision: int = HS_FP64,
                 device: int = 0, stream: int | None = None, refine_tol: float = 0.0, refine_max_iter: int = 0,
                 bm_eta: float = 0.0, leaf_impedance: bool = False):
        self.nL, self.S1, self.S2, self.R = leaves_per_side, S1, S2, R
        self.ctx = hs_create(leaves_per_side, S1, S2, R, precision, device, stream, refine_tol, refine_max_iter,
                             bm_eta, leaf_impedance)

    @property
    def n_nodes(self) -> int:
        return self.nL * self.nL * 256

    def node_coords(self):
        return hs_node_coords(self.ctx, self.n_nodes)

    def build(self, c, k):
        hs_build(self.ctx, c, k)
        return self

    def build_nodes(self, q_nodes, k):
        hs_build_nodes(self.ctx, q_nodes, k)
        return self

    def solve(self, alphas, thetas):
        return hs_solve(self.ctx, alphas, thetas)

    def jacobian(self, alphas, thetas):
        return hs_jacobian(self.ctx, alphas, thetas, self.S1, self.S2)

    def gn_step(self, data, alphas, thetas, lambda_rel, c):
        return hs_gn_step(self.ctx, data, alphas, thetas, lambda_rel, c)

    def gn_step_lsqr(self, data, alphas, thetas, c, mask=None, damp=0.0, tol=1e-3, max_iter=100,
                     products=HS_FP64):
        return hs_gn_step_lsqr(self.ctx, data, alphas, thetas, c, mask, damp, tol, max_iter, products)

    def gradient(self, data, alphas, thetas):
        return hs_gradient(self.ctx, data, alphas, thetas, self.S1, self.S2)

    def launch_count(self) -> int:
        return hs_launch_count(self.ctx)

    def close(self):
        if self.ctx:
            hs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
