"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol include/hs.h declares, and rejects bad arguments before touching CUDA."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hs.h")
DIAG_HEADER = os.path.join(ROOT, "include", "hs_diag.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1608_06871_gb300.build import build
    build()
    import paper_1608_06871_gb300 as hs
    return hs


def declared_functions(path=HEADER):
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hs_[a-z_]+)\s*\(", text)))


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for n in ("hs_create", "hs_build", "hs_solve", "hs_jacobian", "hs_gn_step", "hs_gradient",
              "hs_last_error", "hs_destroy"):
        assert n in names


@pytest.mark.parametrize("path", [HEADER, DIAG_HEADER])
def test_library_exports_every_declared_symbol(lib, path):
    L = lib.lib()
    for name in declared_functions(path):
        assert hasattr(L, name), name


@pytest.mark.parametrize("path", [HEADER, DIAG_HEADER])
def test_binding_covers_every_declared_symbol(lib, path):
    for name in declared_functions(path):
        assert hasattr(lib, name), name


def test_bad_configs_are_rejected_without_a_gpu(lib):
    L = lib.lib()
    ctx = ctypes.c_void_p()
    for kw in (dict(leaves_per_side=3), dict(leaves_per_side=0), dict(S1=0), dict(R=1.0), dict(precision=7),
               dict(bm_eta=-1.0), dict(bm_eta=float("nan")), dict(leaf_impedance=2), dict(leaf_impedance=-1)):
        base = dict(R=3.0, leaves_per_side=4, S1=4, S2=4, precision=0, device=0, stream=None,
                    refine_tol=0.0, refine_max_iter=0, bm_eta=0.0, leaf_impedance=0)
        base.update(kw)
        cfg = lib.hs_config(**base)
        assert L.hs_create(ctypes.byref(ctx), ctypes.byref(cfg)) == lib.HS_EINVAL
        assert not ctx.value
    assert L.hs_create(None, None) == lib.HS_EINVAL


def test_null_context_paths(lib):
    L = lib.lib()
    assert L.hs_last_error(None) == b"NULL context"
    assert L.hs_launch_count(None) == 0
    L.hs_destroy(None)  # no-op
    assert L.hs_build(None, None, 1, 1, 1.0) == lib.HS_EINVAL
