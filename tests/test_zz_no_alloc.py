"""hsolve_apply_noalloc: the substitution sweeps with every temporary taken
from the library's fixed device scratch array, for callers that cannot let
the library allocate (their device memory belongs to another allocator, or
they must avoid the synchronisation cudaMalloc/cudaFree can imply).

The test calls the entry point through the C-ABI twice in a row and checks
each result against hsolve_apply on the same factorization, within the
float64 parity tolerance of the other GPU tests (1e-10 relative), and on a
3D factorization with coarse levels and a dense top of more than 256
unknowns also against the float64 oracle's M^{-1} b; it checks that the
calls leave the device's free memory unchanged and that a request larger
than the fixed array is refused.  It lives in a file that pytest collects
last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1712_07297_gb300 import inputs as I  # noqa: E402
from oracle import hsolver as H  # noqa: E402

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def hs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_07297_gb300 import build
    build.build()
    from paper_1712_07297_gb300 import hsolve
    hsolve.load()
    return hsolve


@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_noalloc_apply_matches_apply_twice(hs, precision):
    p = I.poisson((64, 64))
    s = hs.Solver.from_problem(p, leaf_size=64, symmetric=1)
    s.factor(1e-3, precision)
    b1 = torch.from_numpy(I.rhs(p.n, 2, seed=21)).cuda()
    b2 = torch.from_numpy(I.rhs(p.n, 2, seed=22)).cuda()
    ref1 = s.apply(b1).cpu().numpy()
    ref2 = s.apply(b2).cpu().numpy()
    out = torch.full_like(b1, float("nan"))
    got1 = s.apply_noalloc(b1, out).cpu().numpy()
    assert _rel(got1, ref1) < 1e-10
    out2 = torch.full_like(b2, float("nan"))
    got2 = s.apply_noalloc(b2, out2).cpu().numpy()
    assert _rel(got2, ref2) < 1e-10
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed_fp32", 2e-3)])
def test_noalloc_3d_with_dense_top_matches_oracle(hs, precision, tol):
    # clusters of 128 (the full-size workloads' leaf), coarse levels and a
    # dense top of 1,602 unknowns (its sweeps take the two-kernel backward
    # path); the noalloc call comes first on this factorization
    p = I.poisson((32, 32, 32))
    fac = H.factor(p.rowptr, p.col, p.val, p.coords, 128, 1e-2, symmetric=True, top_size=2048)
    s = hs.Solver.from_problem(p, leaf_size=128, symmetric=1, top_size=2048)
    s.factor(1e-2, precision)
    assert s.stats()["top_size"] > 256
    b = I.rhs(p.n, 3, seed=23)
    bt = torch.from_numpy(b).cuda()
    ref = H.solve(fac, b.T).T
    for _ in range(2):
        out = torch.full_like(bt, float("nan"))
        got = s.apply_noalloc(bt, out).cpu().numpy()
        assert _rel(got, ref) < tol
    assert _rel(got, s.apply(bt).cpu().numpy()) < 1e-10
    s.close()


def test_noalloc_leaves_free_memory_unchanged(hs):
    # the first call on a device may load the library's kernels into device
    # memory (the CUDA runtime's lazy module loading, outside the library's
    # control); later calls must not change the free memory at all
    p = I.poisson((64, 64))
    s = hs.Solver.from_problem(p, leaf_size=64, symmetric=1)
    s.factor(1e-3, "mixed_fp32")
    b = torch.from_numpy(I.rhs(p.n, 4, seed=24)).cuda()
    out = torch.empty_like(b)
    s.apply_noalloc(b, out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        s.apply_noalloc(b, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    s.close()


def test_noalloc_rejects_oversized_request(hs):
    p = I.poisson((64, 64))
    s = hs.Solver.from_problem(p, leaf_size=64, symmetric=1)
    s.factor(1e-3, "fp64")
    nrhs = 1200   # about 3 vectors x 4096 x 8 bytes per right-hand side -> > 32 MiB
    b = torch.zeros((nrhs, p.n), dtype=torch.float64, device="cuda")
    out = torch.zeros_like(b)
    with pytest.raises(hs.HsolveError) as e:
        s.apply_noalloc(b, out)
    assert e.value.code == -7
    assert "33554432" in str(e.value)
    s.close()
