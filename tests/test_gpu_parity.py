"""GPU parity: the CUDA library against the float64 CPU oracle, through the
C-ABI (ctypes binding).

Bars (written out per test):
  * ranks of every cluster at every level: identical (integer work);
  * float64 path: M^{-1} b within 1e-10 relative (2-norm) of the oracle's;
  * mixed float32 path: M^{-1} b within a bound derived from float32
    rounding (see _mixed_bound), and the float64 Krylov solve reaching
    1e-10 relative residual;
  * Krylov solves: ||b - A x|| <= 1e-10 ||b|| recomputed here in float64.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1712_07297_gb300 import inputs as I  # noqa: E402
from oracle import hsolver as H  # noqa: E402

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


def _oracle(p, leaf, eps, top_size=0, max_rank=None, compress=0):
    return H.factor(p.rowptr, p.col, p.val, p.coords, leaf, eps, symmetric=p.symmetric,
                    top_size=top_size, max_rank=max_rank, compress=compress)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _ranks_match(s, fac):
    nlev = 0
    for li, lv in enumerate(fac.levels):
        if lv.top is not None:
            break
        sizes, ranks, _ = s.level(li)
        assert list(sizes) == list(lv.sizes), f"level {li} sizes"
        want = [lv.factors[i].k if i in lv.factors else 0 for i in range(lv.nclu)]
        assert list(ranks) == want, f"level {li} ranks"
        nlev += 1
    return nlev


CASES = [
    # (name, problem, leaf, eps)  -- 2D 64x64 clusters of 64, eps 1e-3 is
    # the small headline workload; the others add 3D, ragged sizes and
    # variable coefficients
    ("poisson2d_64", lambda: I.poisson((64, 64)), 64, 1e-3),
    ("poisson3d_16", lambda: I.poisson((16, 16, 16)), 64, 1e-2),
    ("poisson2d_ragged", lambda: I.poisson((37, 23)), 16, 1e-2),
    ("vcdiff3d_12", lambda: I.vc_diffusion((12, 12, 12), seed=2002), 32, 1e-3),
    ("hcdiff3d_12", lambda: I.high_contrast((12, 12, 12), seed=5), 32, 1e-2),
]


@pytest.mark.parametrize("name,mk,leaf,eps", CASES)
def test_fp64_matches_oracle(hs, name, mk, leaf, eps):
    p = mk()
    fac = _oracle(p, leaf, eps)
    s = hs.Solver.from_problem(p, leaf_size=leaf, symmetric=1)
    s.factor(eps, "fp64")
    assert np.array_equal(s.perm(), fac.perm)
    assert _ranks_match(s, fac) >= 1
    b = I.rhs(p.n, 3, seed=1000)
    ref = H.solve(fac, b.T).T
    out = s.apply(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(out, ref) < 1e-10, _rel(out, ref)
    s.close()


@pytest.mark.parametrize("name,mk,leaf,eps", CASES[:3])
def test_fp64_pcg_converges(hs, name, mk, leaf, eps):
    p = mk()
    s = hs.Solver.from_problem(p, leaf_size=leaf, symmetric=1)
    s.factor(eps, "fp64")
    b = I.rhs(p.n, 2, seed=1000)
    x, info = s.solve(torch.from_numpy(b).cuda(), krylov="pcg", tol=1e-10)
    x = x.cpu().numpy()
    A = p.scipy()
    for c in range(2):
        assert np.linalg.norm(b[c] - A @ x[c]) <= 1e-10 * np.linalg.norm(b[c]) * 1.0001
    assert info.rel_residual <= 1e-10
    s.close()


def test_eps0_is_direct(hs):
    p = I.poisson((9, 10, 11))
    s = hs.Solver.from_problem(p, leaf_size=40, symmetric=1)
    s.factor(0.0, "fp64")
    b = I.rhs(p.n, 1, seed=3)
    out = s.apply(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(out[0], np.linalg.solve(p.dense(), b[0])) < 1e-10
    s.close()


@pytest.mark.parametrize("mk,leaf,eps,top", [
    (lambda: I.convection_diffusion((16, 16, 16), 10.0), 64, 1e-2, 0),
    (lambda: I.convection_diffusion((40, 30), 10.0), 32, 1e-3, 0),
    # the paper's Helmholtz operator at 32 points per wavelength (still
    # definite on this small grid; from 32^3 on it is indefinite), LU path
    (lambda: I.helmholtz((16, 16, 16), I.helmholtz_k2(32.0)), 64, 1e-2, 0),
    # merged dense LU tops above 256 unknowns (575 and 973; the indefinite
    # Helmholtz top interchanges rows)
    (lambda: I.convection_diffusion((20, 20, 20), 10.0), 64, 1e-2, 2000),
    (lambda: I.helmholtz((16, 16, 16), 1.0), 64, 1e-2, 1500),
])
def test_general_matches_oracle(hs, mk, leaf, eps, top):
    # nonsymmetric: pivot orders of the LU factors may legitimately differ on
    # near-ties, so the comparison is on M^{-1} b, which does not depend on them
    p = mk()
    fac = H.factor(p.rowptr, p.col, p.val, p.coords, leaf, eps, symmetric=False, top_size=top)
    s = hs.Solver.from_problem(p, leaf_size=leaf, symmetric=0, top_size=top)
    s.factor(eps, "fp64")
    _ranks_match(s, fac)
    if top:
        assert s.stats()["top_size"] == fac.levels[-1].top["n"] > 256
    b = I.rhs(p.n, 2, seed=1002)
    ref = H.solve(fac, b.T).T
    out = s.apply(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(out, ref) < 1e-10, _rel(out, ref)
    x, info = s.solve(torch.from_numpy(b).cuda(), krylov="gmres", tol=1e-10)
    A = p.scipy()
    xx = x.cpu().numpy()
    for c in range(2):
        assert np.linalg.norm(b[c] - A @ xx[c]) <= 1.0001e-10 * np.linalg.norm(b[c])
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_lu_top_one_cluster(hs, precision):
    # one cluster of 4096 unknowns: the whole matrix is the dense top (Alg. 1),
    # factored by the blocked LU with partial pivoting whose panels span
    # 16-CTA thread-block clusters.  An indefinite Helmholtz matrix (2D,
    # k^2 h^2 = 0.5) makes partial pivoting interchange rows.
    #  * A^{-1} = TRt^T T does not depend on the pivot order: within
    #    C u kappa(A) (normwise backward stability of LU with partial
    #    pivoting, growth included in C = 8) of the exact inverse;
    #  * float64: T = L^{-1} P^T and TRt = U^{-T} element by element within
    #    the same bound (the pivot orders agree: no near-ties at float64
    #    rounding);
    #  * the preconditioner is then a direct solver: FGMRES in one step.
    p = I.helmholtz((64, 64), 0.5)
    fac = H.factor(p.rowptr, p.col, p.val, p.coords, p.n, 1e-2, symmetric=False)
    top = fac.levels[0].top
    assert len(fac.levels) == 1 and top["kind"] == "lu" and top["n"] == p.n
    assert not np.array_equal(top["P"], np.eye(p.n))
    s = hs.Solver.from_problem(p, leaf_size=p.n, symmetric=0)
    s.factor(1e-2, precision)
    assert s.stats()["top_size"] == p.n
    c = s.export_level(0)["clusters"][0]
    A = p.dense()[np.ix_(fac.perm, fac.perm)]
    Ainv = np.linalg.inv(A)
    u = 2.0 ** -53 if precision == "fp64" else 2.0 ** -24
    bound = 8 * u * np.linalg.cond(A)
    err = np.abs(c["TRt"].T @ c["T"] - Ainv).max() / np.abs(Ainv).max()
    assert err <= bound, (err, bound)
    if precision == "fp64":
        op = H.top_operators(top)
        for key in ("T", "TRt"):
            e = np.abs(c[key] - op[key]).max() / np.abs(op[key]).max()
            assert e <= bound, (key, e, bound)
    b = I.rhs(p.n, 2, seed=7)
    x, info = s.solve(torch.from_numpy(b).cuda(), krylov="gmres", tol=1e-10)
    Asp = p.scipy()
    xx = x.cpu().numpy()
    for k in range(2):
        assert np.linalg.norm(b[k] - Asp @ xx[k]) <= 1.0001e-10 * np.linalg.norm(b[k])
    assert info.iterations <= (1 if precision == "fp64" else 4)
    s.close()


def test_top_size_above_the_dense_top_limit_is_rejected(hs):
    # a merged dense top must fit one slot vector of the sweeps in shared
    # memory (24,576 unknowns in float64) and, for a general matrix, the first
    # LU panel in one 16-CTA thread-block cluster (24,816): a larger top_size
    # is an argument error of hsolve_factor, raised before any device work
    p = I.poisson((12, 12))
    s = hs.Solver.from_problem(p, leaf_size=16, symmetric=1, top_size=10 ** 6)
    with pytest.raises(hs.HsolveError) as e:
        s.factor(1e-2, "fp64")
    assert e.value.code == -1
    s.close()
    s = hs.Solver.from_problem(p, leaf_size=16, symmetric=1, top_size=24576)
    s.factor(1e-2, "fp64")  # at the limit: the whole 144-unknown matrix is the top
    assert s.stats()["top_size"] == p.n
    s.close()
    q = I.convection_diffusion((12, 12))
    s = hs.Solver.from_problem(q, leaf_size=16, symmetric=0, top_size=30000)
    for prec in ("fp64", "mixed_fp32"):
        with pytest.raises(hs.HsolveError) as e:
            s.factor(1e-2, prec)
        assert e.value.code == -1
    s.close()


@pytest.mark.parametrize("name,mk,leaf,eps", [
    ("poisson2d_64", lambda: I.poisson((64, 64)), 64, 1e-3),
    ("poisson3d_16", lambda: I.poisson((16, 16, 16)), 64, 1e-2),
    ("vcdiff3d_12", lambda: I.vc_diffusion((12, 12, 12), seed=2002), 32, 1e-3),
    ("convdiff3d_16", lambda: I.convection_diffusion((16, 16, 16), 10.0), 64, 1e-2),
])
def test_randomized_matches_oracle(hs, name, mk, leaf, eps):
    # randomized compression: the sketch G Omega is formed on the device from
    # the same counter-based Rademacher signs the oracle draws
    p = mk()
    fac = _oracle(p, leaf, eps, compress=1)
    s = hs.Solver.from_problem(p, leaf_size=leaf, symmetric=1 if p.symmetric else 0, compress=1)
    s.factor(eps, "fp64")
    assert _ranks_match(s, fac) >= 1
    b = I.rhs(p.n, 2, seed=1000)
    ref = H.solve(fac, b.T).T
    out = s.apply(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(out, ref) < 1e-10, _rel(out, ref)
    s.close()


def _mixed_bound(fac):
    # float32 blocks: each stored operator carries a relative error of a few
    # units of 2^-24 times its condition; the preconditioner output is
    # compared at 2e-3 relative, far above float32 rounding (6e-8) times the
    # modest growth through the levels, and far below the eps-level
    # differences a wrong rank or a dropped term would cause.
    return 2e-3


@pytest.mark.parametrize("name,mk,leaf,eps", CASES[:2])
def test_mixed_fp32_close_and_solves(hs, name, mk, leaf, eps):
    p = mk()
    fac = _oracle(p, leaf, eps)
    s = hs.Solver.from_problem(p, leaf_size=leaf, symmetric=1)
    s.factor(eps, "mixed_fp32")
    b = I.rhs(p.n, 1, seed=1000)
    ref = H.solve(fac, b.T).T
    out = s.apply(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(out, ref) < _mixed_bound(fac), _rel(out, ref)
    x, info = s.solve(torch.from_numpy(b).cuda(), krylov="pcg", tol=1e-10)
    xx = x.cpu().numpy()[0]
    assert np.linalg.norm(b[0] - p.scipy() @ xx) <= 1.0001e-10 * np.linalg.norm(b[0])
    s.close()


def test_single_cluster_and_top(hs):
    # n below the leaf size: one cluster, a dense factor (Alg. 1 "small")
    p = I.poisson((5, 7))
    s = hs.Solver.from_problem(p, leaf_size=64, symmetric=1)
    s.factor(1e-2, "fp64")
    b = I.rhs(p.n, 1, seed=4)
    out = s.apply(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(out[0], np.linalg.solve(p.dense(), b[0])) < 1e-12
    s.close()
    # top_size switch: identical to the oracle with the same switch
    p = I.poisson((20, 20))
    fac = _oracle(p, 16, 1e-2, top_size=150)
    s = hs.Solver.from_problem(p, leaf_size=16, symmetric=1, top_size=150)
    s.factor(1e-2, "fp64")
    b = I.rhs(p.n, 1, seed=5)
    out = s.apply(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(out.T, H.solve(fac, b.T)) < 1e-10
    s.close()


def test_1d_and_fixed_rank(hs):
    p = I.poisson((300,))
    s = hs.Solver.from_problem(p, leaf_size=8, symmetric=1)
    s.factor(1e-1, "fp64")
    b = I.rhs(p.n, 1, seed=6)
    out = s.apply(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(out[0], np.linalg.solve(p.dense(), b[0])) < 1e-10
    s.close()
    p = I.poisson((32, 32))
    fac = _oracle(p, 32, 1e-8, max_rank=4)
    s = hs.Solver.from_problem(p, leaf_size=32, symmetric=1, max_rank=4)
    s.factor(1e-8, "fp64")
    _ranks_match(s, fac)
    b = I.rhs(p.n, 1, seed=6)
    out = s.apply(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(out.T, H.solve(fac, b.T)) < 1e-10
    s.close()


def test_errors_are_reported(hs):
    p = I.poisson((8, 8))
    s = hs.Solver.from_problem(p, leaf_size=16, symmetric=1)
    b = torch.zeros((1, p.n), dtype=torch.float64, device="cuda")
    with pytest.raises(hs.HsolveError) as e:
        s.apply(b)
    assert e.value.code == -9
    s.close()
    # symmetric indefinite matrix declared SPD: the Cholesky pivot check fires
    # (k^2 = 1.3 is no eigenvalue of any 4x4 cluster block, so every A_ss is
    # invertible and the general path applies)
    q = I.helmholtz((8, 8), k2=1.3)
    s = hs.Solver.from_problem(q, leaf_size=16, symmetric=1)
    with pytest.raises(hs.HsolveError) as e:
        s.factor(1e-2, "fp64")
    assert e.value.code == -5
    # the same matrix through the general (LU) path factors and solves
    s.close()
    s = hs.Solver.from_problem(q, leaf_size=16, symmetric=0)
    s.factor(0.0, "fp64")
    bb = I.rhs(q.n, 1, seed=8)
    out = s.apply(torch.from_numpy(bb).cuda()).cpu().numpy()
    assert _rel(out[0], np.linalg.solve(q.dense(), bb[0])) < 1e-9
    s.close()


def test_host_solve_api(hs):
    p = I.poisson((30, 30))
    s = hs.Solver.from_problem(p, leaf_size=32, symmetric=1)
    s.factor(1e-2, "fp64")
    b = I.rhs(p.n, 1, seed=9)[0]
    x, info = s.solve_host(b, krylov="pcg", tol=1e-10)
    assert np.linalg.norm(b - p.scipy() @ x) <= 1.0001e-10 * np.linalg.norm(b)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_cluster_qr_equals_single_cta(hs, precision):
    # the pivoted QR on thread-block clusters (distributed shared memory) and
    # the one-CTA-per-cluster path take the same decisions and produce the
    # same factorization
    p = I.poisson((20, 20, 20))
    b = torch.from_numpy(I.rhs(p.n, 1, seed=31)).cuda()
    outs, ranks = [], []
    for cq in (0, 1):
        s = hs.Solver.from_problem(p, leaf_size=64, symmetric=1, cluster_qr=cq)
        s.factor(1e-2, precision)
        ranks.append([list(s.level(l)[1]) for l in range(s.stats()["levels"])])
        outs.append(s.apply(b).cpu().numpy())
        s.close()
    assert ranks[0] == ranks[1]
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert _rel(outs[1], outs[0]) < tol


@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32", "mixed_tf32"])
def test_dense_top_blocked(hs, precision):
    # a top level of more than 256 unknowns goes to the blocked multi-CTA
    # Cholesky and inverse factor (Alg. 1, dense factor when small enough);
    # sizes not multiples of the 64-wide panels (float64); the float32 modes
    # take the recursive tensor-core (3xTF32) top with 128-wide leaves
    p = I.poisson((16, 16, 16))
    fac = _oracle(p, 64, 1e-2, top_size=2000)
    assert any(lv.top is not None and lv.top["n"] > 256 for lv in fac.levels)
    s = hs.Solver.from_problem(p, leaf_size=64, symmetric=1, top_size=2000)
    s.factor(1e-2, precision)
    top = max(lv.top["n"] for lv in fac.levels if lv.top is not None)
    if precision == "fp64":
        assert s.stats()["top_size"] == top
    else:  # float32 blocks may decide a rank differently near the threshold
        assert abs(s.stats()["top_size"] - top) <= 0.02 * top
    b = I.rhs(p.n, 2, seed=41)
    ref = H.solve(fac, b.T).T
    out = s.apply(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(out, ref) < (1e-10 if precision == "fp64" else 2e-3), _rel(out, ref)
    x, info = s.solve(torch.from_numpy(b).cuda(), krylov="pcg", tol=1e-10)
    xx = x.cpu().numpy()
    for c in range(2):
        assert np.linalg.norm(b[c] - p.scipy() @ xx[c]) <= 1.0001e-10 * np.linalg.norm(b[c])
    s.close()


def _equilibrated(p):
    """S A S with S = diag(|a_ii|)^{-1/2}, and S (the definition the library's
    equilibrate option states)."""
    import dataclasses
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    d = np.zeros(p.n)
    np.add.at(d, rows[rows == p.col], p.val[rows == p.col])
    S = np.where(d != 0, 1.0 / np.sqrt(np.abs(np.where(d != 0, d, 1.0))), 1.0)
    return dataclasses.replace(p, val=p.val * S[rows] * S[p.col]), S


@pytest.mark.parametrize("mk,leaf,eps,sym", [
    (lambda: I.vc_diffusion((16, 16, 16), seed=2002), 64, 1e-2, 1),
    (lambda: I.high_contrast((14, 13, 12), seed=5), 40, 1e-3, 1),
    (lambda: I.convection_diffusion((30, 26), 10.0), 32, 1e-2, 0),
])
def test_equilibrate_matches_oracle(hs, mk, leaf, eps, sym):
    # M^{-1} = S Mh^{-1} S with Mh the oracle's factorization of S A S; ranks
    # are those of S A S
    p = mk()
    q, S = _equilibrated(p)
    fac = H.factor(q.rowptr, q.col, q.val, q.coords, leaf, eps, symmetric=bool(sym))
    s = hs.Solver.from_problem(p, leaf_size=leaf, symmetric=sym, equilibrate=1)
    s.factor(eps, "fp64")
    if sym:
        assert _ranks_match(s, fac) >= 1
    b = I.rhs(p.n, 2, seed=1004)
    ref = S[None, :] * H.solve(fac, (S[None, :] * b).T).T
    out = s.apply(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(out, ref) < 1e-10, _rel(out, ref)
    x, info = s.solve(torch.from_numpy(b).cuda(), krylov="pcg" if sym else "gmres", tol=1e-10)
    A = p.scipy()
    x = x.cpu().numpy()
    for c in range(2):
        assert np.linalg.norm(b[c] - A @ x[c]) <= 1e-10 * np.linalg.norm(b[c]) * 1.0001
    s.close()


# Tensor-core precisions: the Schur-complement products run on tcgen05 with
# TF32, 3xTF32 or BF16 operands (float32 accumulation) and the dense top on
# 3xTF32 products.  Bars: the float64 Krylov solve still reaches 1e-10 (the
# outer iteration recovers the accuracy, Sec. 5) in at most twice the
# float64 iterations plus two, and M^{-1} b stays within the operand
# rounding's reach of the oracle: 3xTF32 as float32 (2e-3), TF32 (10-bit
# mantissa) 3e-2, BF16 (7-bit) 3e-1 -- all far below the O(1) differences a
# wrong rank, block or sign would cause.
TC_BOUND = {"mixed_3xtf32": 2e-3, "mixed_tf32": 3e-2, "mixed_bf16": 3e-1}


@pytest.mark.parametrize("precision", ["mixed_tf32", "mixed_3xtf32", "mixed_bf16"])
@pytest.mark.parametrize("name,mk,leaf,eps,top", [
    ("poisson3d_16", lambda: I.poisson((16, 16, 16)), 64, 1e-2, 600),
    ("poisson2d_64", lambda: I.poisson((64, 64)), 64, 1e-3, 0),
])
def test_tensor_core_precisions(hs, precision, name, mk, leaf, eps, top):
    p = mk()
    fac = _oracle(p, leaf, eps, top_size=top)
    s = hs.Solver.from_problem(p, leaf_size=leaf, symmetric=1, top_size=top)
    s.factor(eps, "fp64")
    b = I.rhs(p.n, 2, seed=1005)
    _, info64 = s.solve(torch.from_numpy(b).cuda(), krylov="pcg", tol=1e-10)
    s.factor(eps, precision)
    ref = H.solve(fac, b.T).T
    out = s.apply(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(out, ref) < TC_BOUND[precision], _rel(out, ref)
    x, info = s.solve(torch.from_numpy(b).cuda(), krylov="pcg", tol=1e-10)
    A = p.scipy()
    x = x.cpu().numpy()
    for c in range(2):
        assert np.linalg.norm(b[c] - A @ x[c]) <= 1.0001e-10 * np.linalg.norm(b[c])
    assert info.iterations <= 2 * info64.iterations + 2, (info.iterations, info64.iterations)
    s.close()


# At ranks forced to the oracle's (hsolve_factor_forced), the float32
# factorization is the oracle's approximation in float32 arithmetic: M^{-1} b
# agrees to 1e-5 relative (float32 rounding, 6e-8 per operation, grown by the
# conditioning of the cluster blocks over the levels) -- the bound the
# float32 blocks are held to -- and the float64 one to 1e-10.  The 10^6
# contrast variable-coefficient case is factored as S A S (the equilibration
# option, and the oracle on S A S): unscaled, its cluster blocks' conditioning
# takes float32 to 7e-5.
@pytest.mark.parametrize("precision,bound", [("fp64", 1e-10), ("mixed_fp32", 1e-5)])
@pytest.mark.parametrize("name,mk,leaf,eps", CASES[:4])
def test_forced_ranks_match_oracle(hs, precision, bound, name, mk, leaf, eps):
    p = mk()
    equil = name.startswith("vcdiff")
    q, S = _equilibrated(p) if equil else (p, np.ones(p.n))
    fac = _oracle(q, leaf, eps)
    ranks = [np.asarray(lv.ranks, dtype=np.int32) for lv in fac.levels if lv.top is None]
    s = hs.Solver.from_problem(p, leaf_size=leaf, symmetric=1, equilibrate=int(equil))
    s.factor_forced(precision, ranks)
    assert _ranks_match(s, fac) >= 1
    b = I.rhs(p.n, 2, seed=1006)
    ref = S[None, :] * H.solve(fac, (S[None, :] * b).T).T
    out = s.apply(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(out, ref) < bound, _rel(out, ref)
    s.close()


def test_float32_noise_floor_matches_the_float64_one(hs):
    # a fill block that is zero in exact arithmetic but nonzero through
    # rounding (2D upwind convection-diffusion, level 1) must not get a rank
    # from the noise: the oracle drops it through its float64 floor (1e-14
    # max |A_ss|), the float32 path through its own (1e-6 max |A_ss|, the
    # float32 rounding level of such a block); both give k = 0 there
    p = I.convection_diffusion((30, 30), 10.0)
    fac = H.factor(p.rowptr, p.col, p.val, p.coords, 32, 1e-3, symmetric=False)
    lv = fac.levels[1]
    noisy = [i for i, cf in lv.factors.items() if cf.k == 0 and cf.ncols_fill > 0]
    assert noisy
    for prec in ("fp64", "mixed_fp32"):
        s = hs.Solver.from_problem(p, leaf_size=32, symmetric=0)
        s.factor(1e-3, prec)
        _, ranks, _ = s.level(1)
        assert all(ranks[i] == 0 for i in noisy), (prec, [int(ranks[i]) for i in noisy])
        s.close()
