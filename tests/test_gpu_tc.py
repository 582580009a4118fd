"""The tensor-core product (hsolve_tc_gemm: tcgen05, TF32 / 3xTF32 / BF16
operands, float32 accumulation) against float64 products of the same float32
inputs, through the C-ABI.

Bar, per element: |C - C_ref| <= (2 u_op + (K + 2) 2^-24) (|A| |B|^T)_ij with
u_op the operand rounding unit (TF32: 2^-11, 3xTF32: 2^-21 -- the dropped
lo*lo term and the rounding of lo --, BF16: 2^-8), times 1.5; tiles, ragged
edges, strides of both layouts, alpha/beta and the lower-triangle mode are
covered, and TF32 must be measurably less accurate than 3xTF32 (the tensor
path is the one that ran)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

U_OP = {"tf32": 2.0 ** -11, "3xtf32": 2.0 ** -21, "bf16": 2.0 ** -8}


@pytest.fixture(scope="module")
def hs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_07297_gb300 import build
    build.build()
    from paper_1712_07297_gb300 import hsolve
    hsolve.load()
    return hsolve


def _mat(r, c, layout, g):
    x = torch.rand((r, c), generator=g, dtype=torch.float32) * 2 - 1
    if layout == "col":
        return x.t().contiguous().t().cuda()  # stride (1, r)
    return x.cuda()                             # stride (c, 1)


def _colmajor(m, n, g):
    return (torch.rand((n, m), generator=g, dtype=torch.float32) * 2 - 1).cuda().t()


def _check(hs, mode, M, N, K, la, lb, alpha=1.0, beta=0.0, lower=False, seed=0):
    g = torch.Generator().manual_seed(seed)
    A = _mat(M, K, la, g)
    B = _mat(N, K, lb, g)
    C0 = _colmajor(M, N, g)
    C = C0.clone().t().contiguous().t()
    hs.tc_gemm(mode, A, B, C, alpha=alpha, beta=beta, lower=lower)
    A64, B64, C64 = A.double().cpu(), B.double().cpu(), C0.double().cpu()
    ref = alpha * (A64 @ B64.T) + beta * C64
    scale = abs(alpha) * (A64.abs() @ B64.abs().T) + abs(beta) * C64.abs()
    tol = 1.5 * (2 * U_OP[mode] + (K + 2) * 2.0 ** -24) * scale + 1e-30
    got = C.double().cpu()
    if lower:
        mask = torch.tril(torch.ones(M, N, dtype=torch.bool))
        assert torch.equal(got[~mask], C64[~mask])  # untouched above the diagonal
        err = (got - ref).abs()[mask]
        t = tol[mask]
    else:
        err, t = (got - ref).abs(), tol
    assert bool((err <= t).all()), (mode, M, N, K, float((err / t).max()))
    return float((got - ref).abs().max())


@pytest.mark.parametrize("mode", ["tf32", "3xtf32", "bf16"])
@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (128, 128, 256), (200, 77, 45),
                                   (300, 260, 300), (1, 5, 3), (129, 257, 1000)])
def test_tc_gemm_shapes(hs, mode, M, N, K):
    _check(hs, mode, M, N, K, "col", "col", seed=M + N + K)


@pytest.mark.parametrize("mode", ["tf32", "3xtf32", "bf16"])
@pytest.mark.parametrize("la,lb", [("row", "row"), ("col", "row"), ("row", "col")])
def test_tc_gemm_layouts(hs, mode, la, lb):
    _check(hs, mode, 190, 140, 70, la, lb, seed=7)


@pytest.mark.parametrize("mode", ["tf32", "3xtf32"])
def test_tc_gemm_alpha_beta_lower(hs, mode):
    _check(hs, mode, 300, 300, 96, "col", "col", alpha=-1.0, beta=1.0, lower=True, seed=3)
    _check(hs, mode, 150, 90, 64, "col", "row", alpha=0.5, beta=-2.0, seed=4)


def test_tf32_less_accurate_than_3xtf32(hs):
    e1 = _check(hs, "tf32", 256, 256, 512, "col", "col", seed=11)
    e3 = _check(hs, "3xtf32", 256, 256, 512, "col", "col", seed=11)
    assert e3 < e1 / 50, (e1, e3)


def test_tc_gemm_k0_scales_c(hs):
    # K = 0: the product is empty; C = beta C
    _check(hs, "tf32", 64, 64, 0, "col", "col", beta=0.25, seed=5)
