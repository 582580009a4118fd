"""The serving runtime (hsolve_server_*) through the C-ABI: continuous
batching of requests of several matrices, a device memory budget with
eviction, and results that do not depend on the batch they were served in.

Bars: every request's solution reaches the stated relative residual
(recomputed here in float64); each equals the solution of its right-hand
sides solved alone on a separate handle with the same settings to 1e-12
relative (the batched Krylov iterations treat columns independently, so the
two agree to rounding, in practice bit for bit); the budget forces evictions
and refactorizations without changing any result."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1712_07297_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu

FAMS = {
    "p2d": (lambda: I.poisson((32, 32)), 64, 1e-2),
    "p3d": (lambda: I.poisson((12, 12, 12)), 64, 1e-2),
    "hc3d": (lambda: I.high_contrast((12, 11, 10), seed=5), 40, 1e-2),
}


@pytest.fixture(scope="module")
def hs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_07297_gb300 import build
    build.build()
    from paper_1712_07297_gb300 import hsolve
    hsolve.load()
    return hsolve


def _solo(hs, p, leaf, eps, b):
    s = hs.Solver.from_problem(p, leaf_size=leaf, symmetric=1)
    s.factor(eps, "mixed_fp32")
    x, _ = s.solve(torch.from_numpy(b).cuda(), krylov="pcg", tol=1e-10, maxit=500)
    s.close()
    return x.cpu().numpy()


def _run(hs, budget, nreq, seed):
    rng = np.random.default_rng(seed)
    probs = {k: v[0]() for k, v in FAMS.items()}
    srv = hs.Server(memory_budget=budget, max_batch_rhs=24, workers=3)
    ids = {k: srv.add_matrix(probs[k], FAMS[k][2], "mixed_fp32", "pcg", 1e-10, 500,
                             leaf_size=FAMS[k][1], symmetric=1) for k in FAMS}
    reqs = []
    for i in range(nreq):
        fam = list(FAMS)[rng.integers(0, len(FAMS))]
        b = I.rhs(probs[fam].n, int(rng.integers(1, 7)), seed=seed * 1000 + i)
        reqs.append((fam, b, srv.submit(ids[fam], b)))
        if i % 7 == 6:
            time.sleep(0.01)  # arrivals while batches run
    out = [(fam, b) + srv.wait(t) for fam, b, t in reqs]
    st = srv.stats()
    srv.close()
    return probs, out, st


def test_serving_results_match_solo(hs):
    probs, out, st = _run(hs, budget=0, nreq=30, seed=1)
    assert st["requests_done"] == 30 and st["factorizations"] == 3
    assert st["batches"] < 30  # some requests shared a batch
    assert any(r["batch_rhs"] > b.shape[0] for _, b, _, r in out)
    for fam, b, x, r in out:
        p = probs[fam]
        A = p.scipy()
        assert r["status"] == 0 and r["latency_ms"] >= r["service_ms"] >= 0
        for c in range(b.shape[0]):
            assert np.linalg.norm(b[c] - A @ x[c]) <= 1.0001e-10 * np.linalg.norm(b[c])
        xs = _solo(hs, p, FAMS[fam][1], FAMS[fam][2], b)
        assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs), fam


def test_serving_budget_evicts(hs):
    # a budget below the three factorizations together: matrices are
    # evicted and factored again, results unchanged
    probs, out, st = _run(hs, budget=1, nreq=18, seed=2)
    assert st["requests_done"] == 18
    assert st["evictions"] > 0 and st["factorizations"] > 3
    for fam, b, x, r in out:
        A = probs[fam].scipy()
        for c in range(b.shape[0]):
            assert np.linalg.norm(b[c] - A @ x[c]) <= 1.0001e-10 * np.linalg.norm(b[c])
