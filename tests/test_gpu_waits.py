"""The library's bounded device wait (the mbarrier wait of the tensor-core
kernels) gives up and reports instead of hanging: it runs once on a barrier
nothing arrives at, with a short limit (hsolve_wait_selftest), and must
return HSOLVE_ERR_TIMEOUT; the device stays usable for a factorization and
solve afterwards."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1712_07297_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_07297_gb300 import build
    build.build()
    from paper_1712_07297_gb300 import hsolve
    hsolve.load()
    return hsolve


@pytest.mark.parametrize("kind", ["mbarrier"])
def test_bounded_wait_times_out(hs, kind):
    # 100,000 SM clocks: about 50 microseconds
    assert hs.wait_selftest(kind, 100000) == -8
    # the context is intact: a small factorization and solve still work
    p = I.poisson((16, 16))
    s = hs.Solver.from_problem(p, leaf_size=16, symmetric=1)
    s.factor(1e-2, "mixed_fp32")
    b = torch.from_numpy(I.rhs(p.n, 1, seed=9)).cuda()
    x, info = s.solve(b, krylov="pcg", tol=1e-10)
    r = p.scipy() @ x.cpu().numpy()[0] - b.cpu().numpy()[0]
    assert np.linalg.norm(r) <= 1.0001e-10 * np.linalg.norm(b.cpu().numpy()[0])
    s.close()


def test_wait_selftest_arguments(hs):
    assert hs.wait_selftest.__doc__
    lib = hs.load()
    assert lib.hsolve_wait_selftest(1, 1000, None) == -1
    assert lib.hsolve_wait_selftest(0, -1, None) == -1
