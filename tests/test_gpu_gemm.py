"""The library's FP64 complex GEMM (`hs_zgemm`): the kernels of the FP64
solver and of the mixed path's FP64 refinement, including the split-k
reduction across thread-block clusters.  Checked entry by entry against a
plain PyTorch complex128 product on the host within the componentwise bound
|C - AB| <= 2 k u (|A||B|), u = 2**-53, and for bitwise reproducibility."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module")
def hs():
    from paper_1608_06871_gb300.build import build
    build()
    import paper_1608_06871_gb300 as mod
    return mod


def _rand(shape, g):
    return torch.complex(torch.randn(shape, generator=g, dtype=torch.float64),
                         torch.randn(shape, generator=g, dtype=torch.float64))


# (transA, transB, m, n, k): the exterior residual (1792 x 128 x 1792, split k),
# the far field (op = T, 128 x 256 x 3584), a 64-tile shape and ragged tails
CASES = [(False, False, 1792, 128, 1792), (True, True, 128, 256, 3584), (False, False, 640, 576, 320),
         (False, True, 77, 45, 300), (True, False, 33, 129, 513), (False, False, 5, 3, 2)]


@pytest.mark.parametrize("tA,tB,m,n,k", CASES)
@pytest.mark.parametrize("acc", [False, True])
def test_zgemm_vs_torch(hs, tA, tB, m, n, k, acc):
    g = torch.Generator().manual_seed(m * 31 + n * 7 + k)
    A = _rand((k, m) if tA else (m, k), g)
    B = _rand((n, k) if tB else (k, n), g)
    C0 = _rand((m, n), g)
    opA = A.T if tA else A
    opB = B.T if tB else B
    ref = opA @ opB + (C0 if acc else 0)
    bound = 2 * k * U * (opA.abs() @ opB.abs() + (C0.abs() if acc else 0))
    dC = C0.cuda().contiguous()
    hs.hs_zgemm(A.cuda().contiguous(), B.cuda().contiguous(), dC, tA, tB, acc)
    got = dC.cpu()
    assert bool(((got - ref).abs() <= bound).all()), float(((got - ref).abs() / bound).max())


def test_zgemm_split_k_reproducible(hs):
    g = torch.Generator().manual_seed(9)
    A, B = _rand((1792, 1792), g).cuda(), _rand((1792, 128), g).cuda()
    outs = []
    for _ in range(3):
        C = torch.zeros((1792, 128), dtype=torch.complex128, device="cuda")
        hs.hs_zgemm(A, B, C)
        outs.append(C.cpu())
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
