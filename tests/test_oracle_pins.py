"""Pins for the CPU oracle (no GPU).

Each test ties the oracle to something other than itself: a dense direct
solve (library LU), closed-form Laplacian spectra, LAPACK's pivoted QR, the
structural fill-in property of Sec. 2.3, a literal N x N restatement of Eqs.
scaling/elim/perm, or an invariant of the method.  The paper prints no worked
numerical example, so no value here comes from its text.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from paper_1712_07297_gb300 import inputs as I
from oracle import hsolver as H
from oracle import krylov as K
from oracle import matrix_form as MF


def _fac(p, leaf, eps, **kw):
    # Cholesky path for SPD problems, LU (two-sided) otherwise
    return H.factor(p.rowptr, p.col, p.val, p.coords, leaf, eps, symmetric=p.spd, **kw)


def _minv(p, leaf, eps, **kw):
    return H.solve(_fac(p, leaf, eps, **kw), np.eye(p.n))


SMALL = [
    (lambda: I.poisson((12, 12)), 9),
    (lambda: I.poisson((6, 6, 6)), 14),
    (lambda: I.vc_diffusion((6, 6, 6), seed=4), 14),
    (lambda: I.convection_diffusion((6, 6, 6), 10.0), 14),
    (lambda: I.convection_diffusion((12, 12), 10.0), 9),
    (lambda: I.high_contrast((8, 8, 8), seed=2), 16),
    # symmetric indefinite: -Lap - k^2 with k^2 h^2 = 2 (several negative
    # eigenvalues on this grid), through the LU path
    (lambda: I.helmholtz((6, 6, 6), 2.0), 14),
]


@pytest.mark.parametrize("mk,leaf", SMALL)
def test_eps0_is_a_direct_solver(mk, leaf):
    # Sec. 2.2 / Alg. 1: without truncation the factorization is exact.
    p = mk()
    b = I.rhs(p.n, 3, seed=11).T
    x = H.solve(_fac(p, leaf, 0.0), b)
    xr = np.linalg.solve(p.dense(), b)
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-10


def test_eps0_eigenvector_closed_form():
    shape = (10, 12)
    p = I.poisson(shape)
    idx = (3, 5)
    v = np.ones(p.n)
    lam = 0.0
    for d, s in enumerate(shape):
        v *= np.sin(idx[d] * np.pi * (p.coords[:, d] + 1) / (s + 1))
        lam += 4 * np.sin(idx[d] * np.pi / (2 * (s + 1))) ** 2
    x = H.solve(_fac(p, 8, 0.0), v)
    np.testing.assert_allclose(x, v / lam, atol=1e-12 * np.abs(v / lam).max())


@pytest.mark.parametrize("eps", [1e-1, 1e-2])
def test_1d_laplacian_exact_for_any_eps(eps):
    # In 1-D every cluster's neighbours are eliminated before fill can reach
    # it in (colour, index) order, so nothing is dropped: M^{-1} = A^{-1}
    # and the spectrum of M^{-1} is 1 / (4 sin^2(j pi / (2 (n+1)))).
    n = 40
    p = I.poisson((n,))
    fac = _fac(p, 4, eps)
    Minv = H.solve(fac, np.eye(n))
    np.testing.assert_allclose(Minv @ p.dense(), np.eye(n), atol=1e-12)
    lam = 4 * np.sin(np.arange(1, n + 1) * np.pi / (2 * (n + 1))) ** 2
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh((Minv + Minv.T) / 2)), np.sort(1 / lam), rtol=1e-10)


@pytest.mark.parametrize("mk,leaf", SMALL[:4])
def test_error_falls_with_eps(mk, leaf):
    # Sec. 5.3: a smaller truncation error gives a better preconditioner.
    p = mk()
    A = p.dense()
    errs = []
    for eps in [3e-1, 1e-2, 1e-4, 1e-7, 0.0]:
        errs.append(np.linalg.norm(np.eye(p.n) - _minv(p, leaf, eps) @ A, 2))
    assert all(errs[i + 1] <= errs[i] * 1.05 for i in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-10 and errs[0] > 1e3 * errs[-2]


def test_pcg_iterations_fall_with_eps():
    p = I.poisson((8, 8, 8))
    A = p.scipy()
    b = I.rhs(p.n, 1, seed=3)[0]
    its = []
    for eps in [3e-1, 1e-2, 1e-4, 0.0]:
        fac = _fac(p, 16, eps)
        _, it, res = K.pcg(A, b, lambda r: H.solve(fac, r), tol=1e-10)
        assert res <= 1e-10
        its.append(it)
    assert its == sorted(its, reverse=True) and its[-1] <= 2 and its[0] > its[-1]


def test_spd_preconditioner_is_symmetric():
    p = I.poisson((6, 6, 6))
    M = _minv(p, 14, 1e-2)
    np.testing.assert_allclose(M, M.T, atol=1e-13 * np.abs(M).max())
    assert np.linalg.eigvalsh((M + M.T) / 2).min() > 0


def test_householder_convention():
    rng = np.random.default_rng(1)
    for x in [rng.standard_normal(7), -np.abs(rng.standard_normal(5)), np.array([0.0, 3.0, 4.0]),
              np.array([-2.0, 0.0, 0.0])]:
        v, tau, beta = H.householder(x)
        Hm = np.eye(len(x)) - tau * np.outer(v, v)
        e = np.zeros(len(x))
        e[0] = beta
        np.testing.assert_allclose(Hm @ x, e, atol=1e-14 * np.linalg.norm(x))
        np.testing.assert_allclose(Hm @ Hm.T, np.eye(len(x)), atol=1e-14)
        assert abs(beta) == pytest.approx(np.linalg.norm(x))
        assert (beta < 0) == (x[0] >= 0)


def test_cpqr_matches_lapack_pivoting():
    rng = np.random.default_rng(5)
    G = rng.standard_normal((30, 50)) * np.logspace(0, -3, 50)[rng.permutation(50)]
    cp = H.cpqr(G, 1e-2)
    Q, R, P = sla.qr(G, pivoting=True)
    k = cp["k"]
    assert list(P[:k]) == cp["piv"]
    np.testing.assert_allclose(cp["rdiag"], np.abs(np.diag(R))[:k], rtol=1e-12)
    # truncation rule |r_kk| <= eps |r_11| at the first excluded step
    d = np.abs(np.diag(R))
    assert d[k - 1] > 1e-2 * d[0] >= d[k]
    U = cp["U"]
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-13)
    np.testing.assert_allclose(U @ U.T, Q[:, :k] @ Q[:, :k].T, atol=1e-12)


def test_cpqr_rank_follows_singular_value_gap():
    rng = np.random.default_rng(9)
    X, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    Y, _ = np.linalg.qr(rng.standard_normal((90, 40)))
    s = np.array([1.0, 0.7, 0.4, 0.2] + [1e-9] * 36)
    G = X @ np.diag(s) @ Y.T
    cp = H.cpqr(G, 1e-4)
    assert cp["k"] == 4
    # U spans the dominant left singular subspace
    np.testing.assert_allclose(cp["U"] @ cp["U"].T, X[:, :4] @ X[:, :4].T, atol=1e-7)
    assert H.cpqr(G, 0.0)["k"] == 40
    assert H.cpqr(G, 1e-4, max_rank=2)["k"] == 2


def test_cpqr_ties_go_to_lowest_index():
    G = np.zeros((4, 4))
    G[1, 0] = 2.0
    G[0, 1] = -2.0
    G[2, 2] = 2.0
    G[3, 3] = 1.0
    cp = H.cpqr(G, 0.1)
    assert cp["piv"][:3] == [0, 1, 2]
    assert cp["k"] == 4


def test_complement_is_orthogonal():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((20, 6))
    V = H.complement(X)
    assert V.shape == (20, 14)
    np.testing.assert_allclose(V.T @ X, 0, atol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(14), atol=1e-13)


@pytest.mark.parametrize("mk,leaf,eps", [
    (lambda: I.poisson((12, 12)), 9, 1e-2),
    (lambda: I.poisson((6, 6, 6)), 14, 1e-2),
    (lambda: I.vc_diffusion((6, 6, 6), seed=4), 14, 1e-3),
    (lambda: I.convection_diffusion((12, 12), 10.0), 9, 1e-2),
])
def test_block_oracle_equals_matrix_form(mk, leaf, eps):
    # Eqs. scaling/elim/perm applied as N x N operators with the Eq. lra
    # replacement made explicit give the same preconditioner; after each
    # W_s the fine block is I (Eq. elim), the fine DOFs are decoupled from the
    # coarse and far ones, and no nonzero block lies beyond distance two
    # (Sec. 2.3: level-2 fill-in is never created).
    p = mk()
    r = MF.factor_dense(p.dense(), p.coords, leaf, eps, symmetric=p.symmetric)
    Mb = _minv(p, leaf, eps)
    assert np.abs(Mb - r["Minv"]).max() <= 1e-12 * np.abs(Mb).max()
    c = r["checks"]
    assert c["outside_d2"] == 0.0
    assert c["fine_identity"] < 1e-10 and c["fine_decoupled"] < 1e-10 and c.get("fine_far", 0) < 1e-12
    assert c["final_identity"] < 1e-10


def test_colouring_is_distance_two():
    p = I.poisson((16, 16, 16))
    fac = _fac(p, 32, 1e-2)
    for lv in fac.levels[:-1]:
        for i in range(lv.nclu):
            for j in lv.adj[i] | lv.d2[i]:
                assert lv.colour[i] != lv.colour[j]
        assert lv.order == sorted(range(lv.nclu), key=lambda i: (lv.colour[i], i))


def test_rcb_boxes():
    p = I.poisson((8, 8))
    depth, leaves = H.rcb_leaves(p.coords, 8)
    assert depth == 3 and len(leaves) == 8
    for lf in leaves:
        c = p.coords[lf]
        ext = tuple(c.max(0) - c.min(0) + 1)
        assert ext == (2, 4)       # x, y, x splits: 8x8 -> 4x8 -> 4x4 -> 2x4
    p3 = I.poisson((16, 16, 16))
    _, lv3 = H.rcb_leaves(p3.coords, 128)
    assert len(lv3) == 32
    assert {tuple(p3.coords[l].max(0) - p3.coords[l].min(0) + 1) for l in lv3} == {(4, 4, 8)}
    assert np.array_equal(np.sort(np.concatenate(lv3)), np.arange(p3.n))


def test_no_fill_cluster_is_block_cholesky():
    # Sec. 2.2: with no fill-in, E_s = I and W_s is one block-Cholesky step.
    p = I.poisson((12, 12))
    fac = _fac(p, 9, 1e-2)
    lv = fac.levels[0]
    A = p.dense()[np.ix_(fac.perm, fac.perm)]
    s = lv.order[0]
    cf = lv.factors[s]
    assert cf.k == 0 and cf.TL is None
    o = lv.offsets
    S = slice(o[s], o[s + 1])
    N = np.concatenate([np.arange(o[n], o[n + 1]) for n, _ in cf.nbrs])
    Ass, AsN = A[S, S], A[S][:, N]
    np.testing.assert_allclose(cf.LF @ cf.LF.T, Ass, atol=1e-13)
    np.testing.assert_allclose(cf.BR.T @ cf.BR, AsN.T @ np.linalg.solve(Ass, AsN), atol=1e-13)


def test_fixed_rank_caps_ranks():
    p = I.poisson((16, 16))
    fac = _fac(p, 16, 1e-6, max_rank=3)
    assert max(f.k for f in fac.levels[0].factors.values()) <= 3


@pytest.mark.parametrize("mk", [lambda: I.poisson((12, 12)),
                                lambda: I.convection_diffusion((12, 12)),
                                lambda: I.helmholtz((6, 6, 6), 2.0)])
def test_dense_top_switch(mk):
    # Alg. 1's "small enough" test is a size test for SPD and general
    # matrices alike: a level of at most top_size unknowns is factored
    # densely (Cholesky, or LU with partial pivoting), and that dense factor
    # is exact
    p = mk()
    b = I.rhs(p.n, 1, seed=1)[0]
    fac = _fac(p, 9, 0.0, top_size=10 ** 9)   # one dense factor
    assert len(fac.levels) == 1
    assert fac.levels[0].top["kind"] == ("chol" if p.spd else "lu")
    np.testing.assert_allclose(p.scipy() @ H.solve(fac, b), b, atol=1e-11)
    # a mid-hierarchy top: the level it is taken at is the first one of at
    # most top_size unknowns
    full = _fac(p, 9, 0.0)
    sizes = [int(lv.offsets[-1]) for lv in full.levels]
    cut = sizes[1]
    fac = _fac(p, 9, 0.0, top_size=cut)
    assert len(fac.levels) == 2 and fac.levels[1].top["n"] == cut
    np.testing.assert_allclose(p.scipy() @ H.solve(fac, b), b, atol=1e-10)


def test_lu_top_operators():
    # A = P L U: T = L^{-1} P^T and TRt = U^{-T} give A^{-1} = TRt^T T, L is
    # unit lower, and on an indefinite matrix partial pivoting bounds every
    # multiplier by 1 (and does interchange rows)
    p = I.helmholtz((6, 6, 6), 2.0)
    fac = H.factor(p.rowptr, p.col, p.val, p.coords, 9, 0.0, symmetric=False, top_size=10 ** 9)
    top = fac.levels[0].top
    op = H.top_operators(top)
    A = p.dense()[np.ix_(fac.perm, fac.perm)]
    np.testing.assert_allclose(op["TRt"].T @ op["T"] @ A, np.eye(p.n), atol=1e-10)
    L = top["L"]
    np.testing.assert_array_equal(np.diag(L), 1.0)
    assert np.abs(L).max() <= 1.0 + 1e-15
    assert not np.array_equal(top["P"], np.eye(p.n))
    assert np.allclose(np.triu(op["T"] @ top["P"], 1), 0.0)


@pytest.mark.parametrize("method", ["pcg", "gmres"])
def test_krylov_against_direct(method):
    p = I.poisson((10, 10)) if method == "pcg" else I.convection_diffusion((10, 10))
    A = p.scipy()
    b = I.rhs(p.n, 1, seed=2)[0]
    fn = K.pcg if method == "pcg" else (lambda *a, **k: K.fgmres(*a, restart=20, **k))
    x, it, res = fn(A, b, lambda r: r, tol=1e-10, maxit=2000)
    np.testing.assert_allclose(x, np.linalg.solve(p.dense(), b), rtol=1e-8, atol=1e-9)
    assert res <= 1e-10 and it > 5
    fac = _fac(p, 9, 0.0)
    x1, it1, res1 = fn(A, b, lambda r: H.solve(fac, r), tol=1e-10)
    assert it1 <= 2 and res1 <= 1e-10


def test_noise_floor_drops_rounding_level_fill():
    # A fill block at the rounding level of the cluster's diagonal block is
    # zero in exact arithmetic: its "rank" must not be decided by noise.
    rng = np.random.default_rng(3)
    G = rng.standard_normal((10, 30))
    assert H.cpqr(1e-20 * G, 1e-3, floor=1e-14)["k"] == 0
    assert H.cpqr(1e-20 * G, 1e-3)["k"] == 10
    assert H.cpqr(G, 1e-3, floor=1e-14)["k"] == 10
    # 2D upwind convection-diffusion makes such a block at level 1: its fill
    # columns are nonzero, yet no direction survives (k = 0 with a nonzero
    # block is only possible through the floor, since |r_11| > eps |r_11|)
    p = I.convection_diffusion((30, 30), 10.0)
    fac = _fac(p, 32, 1e-3)
    assert any(cf.k == 0 and cf.ncols_fill > 0 for cf in fac.levels[1].factors.values())
    b = I.rhs(p.n, 1, seed=1)[0]
    x = H.solve(_fac(p, 32, 0.0), b)
    np.testing.assert_allclose(p.scipy() @ x, b, atol=1e-11)


def test_splitmix64_reference_output():
    # SplitMix64's published reference stream seeded with 0 starts 0xe220a8397b1dcdaf
    assert int(H.splitmix64(np.uint64(0))) == 0xE220A8397B1DCDAF
    Om = H.sketch_matrix(50, 20)
    np.testing.assert_array_equal(np.abs(Om), 1 / np.sqrt(20))
    assert abs(Om.mean()) < 0.1 and np.abs(Om.T @ Om - np.eye(20) * 50 / 20).max() < 5


@pytest.mark.parametrize("mk,leaf", SMALL)
def test_randomized_eps0_is_direct(mk, leaf):
    p = mk()
    b = I.rhs(p.n, 1, seed=12)[0]
    x = H.solve(_fac(p, leaf, 0.0, compress=1), b)
    np.testing.assert_allclose(p.scipy() @ x, b, atol=1e-9 * np.abs(b).max())


def test_randomized_ranks_close_and_quality():
    # the sketch keeps the rank profile close to the exact pivoted QR's and
    # the preconditioner quality comparable (Sec. 5.3 trend holds too)
    p = I.poisson((8, 8, 8))
    A = p.dense()
    e_ex, e_rd = [], []
    for eps in [1e-1, 1e-2, 1e-4]:
        fe = _fac(p, 16, eps, compress=0)
        fr = _fac(p, 16, eps, compress=1)
        ke = sum(f.k for f in fe.levels[0].factors.values())
        kr = sum(f.k for f in fr.levels[0].factors.values())
        assert abs(ke - kr) <= 0.35 * ke + 4
        e_ex.append(np.linalg.norm(np.eye(p.n) - H.solve(fe, np.eye(p.n)) @ A, 2))
        e_rd.append(np.linalg.norm(np.eye(p.n) - H.solve(fr, np.eye(p.n)) @ A, 2))
    assert e_rd == sorted(e_rd, reverse=True)
    assert all(r < 30 * e for r, e in zip(e_rd, e_ex))


def test_smallest_last_order_by_definition():
    # brute force on a random graph: remove, one at a time, the remaining
    # vertex of fewest remaining neighbours (ties: lowest index); the order is
    # the reverse of the removals; then every colour class is independent in
    # the distance-<=2 graph and no colour exceeds the greedy bound
    rng = np.random.default_rng(11)
    n = 60
    adj = [set() for _ in range(n)]
    for _ in range(150):
        a, b = rng.integers(0, n, 2)
        if a != b:
            adj[a].add(int(b))
            adj[b].add(int(a))
    d2 = H.distance2(adj)
    nb = [adj[i] | d2[i] for i in range(n)]
    rem, removed = set(range(n)), []
    while rem:
        i = min(rem, key=lambda v: (len(nb[v] & rem), v))
        removed.append(i)
        rem.discard(i)
    assert H.smallest_last_order(adj, d2) == removed[::-1]
    col = H.greedy_colour(adj, d2)
    for i in range(n):
        assert all(col[i] != col[j] for j in nb[i])
        assert col[i] <= len(nb[i])


# ---------------------------------------------------------------------------
# The stored operators (the form the library exports, Eqs. scaling + elim)
# ---------------------------------------------------------------------------

def _stored_cases():
    return [
        (I.poisson((20, 20)), 16, 1e-2, True),
        (I.poisson((8, 8, 8)), 32, 1e-2, True),
        (I.convection_diffusion((14, 12), 10.0), 16, 1e-2, False),
    ]


@pytest.mark.parametrize("case", range(3))
def test_stored_operators_block_diagonalise(case):
    # T' A_ss T'_R = diag(C, I_f) with C = U^T A_ss^{-1} U: the sparsification
    # operator decouples coarse from fine unknowns (V^T A_ss^{-1} U = 0) and
    # the folded factors of F turn the fine block into the identity
    p, leaf, eps, sym = _stored_cases()[case]
    fac = H.factor(p.rowptr, p.col, p.val, p.coords, leaf, eps, symmetric=sym)
    seen = 0
    for lv in fac.levels:
        if lv.top is not None:
            op = H.top_operators(lv.top)
            if op is not None:
                A = (lv.top["L"] @ lv.top["L"].T if lv.top["kind"] == "chol"
                     else lv.top["P"] @ lv.top["L"] @ lv.top["U"])
                TR = op["T"].T if op["TRt"] is None else op["TRt"].T
                assert np.abs(op["T"] @ A @ TR - np.eye(lv.top["n"])).max() < 1e-12
            continue
        for cf in lv.factors.values():
            op = H.stored_operators(cf, sym)
            if op is None:
                continue
            T = op["T"]
            TR = T.T if sym else op["TRt"].T
            k, f = cf.k, cf.m - cf.k
            D = T @ cf.Ass @ TR
            if cf.TL is None:  # k = 0: no coarse block
                C = np.zeros((0, 0))
            else:
                C = cf.TL[:k] @ cf.Ass @ (cf.TL[:k].T if sym else cf.TR[:, :k])
            scale = max(np.abs(D).max(), 1.0)
            assert np.abs(D[:k, :k] - C).max(initial=0) <= 1e-12 * scale
            assert np.abs(D[:k, k:]).max(initial=0) <= 1e-12 * scale
            assert np.abs(D[k:, :k]).max(initial=0) <= 1e-12 * scale
            assert np.abs(D[k:, k:] - np.eye(f)).max(initial=0) <= 1e-12 * scale
            assert np.array_equal(op["Y"][k:], cf.BR)
            seen += 1
    assert seen > 3


@pytest.mark.parametrize("case", range(3))
def test_stored_operators_reproduce_the_solve(case):
    # Alg. 2 written with the stored operators only (forward z_s = T' y_s,
    # y_N -= (B_L rows) z_f; backward z_f = x_f - B_R x_N, x_s = T'_R z)
    # must give the oracle's M^{-1} b: a transposed, permuted or dropped piece
    # of T', T'_R, Y or X^T changes the result
    p, leaf, eps, sym = _stored_cases()[case]
    fac = H.factor(p.rowptr, p.col, p.val, p.coords, leaf, eps, symmetric=sym)
    b = I.rhs(p.n, 2, seed=11).T
    ref = H.solve(fac, b)
    y = b[fac.perm].copy()
    stack = []
    for lv in fac.levels:
        if lv.top is not None:
            op = H.top_operators(lv.top)
            if op is not None:
                z = op["T"] @ y
                y = (op["T"].T if op["TRt"] is None else op["TRt"].T) @ z
            break
        for s in lv.order:
            cf = lv.factors.get(s)
            op = None if cf is None else H.stored_operators(cf, sym)
            if op is None:
                continue
            o = lv.offsets[s]
            z = op["T"] @ y[o:o + cf.m]
            BLt = (op["Y"] if sym else op["XT"])[cf.k:]
            c0 = 0
            for n, w in cf.nbrs:
                on = lv.offsets[n]
                y[on:on + w] -= BLt[:, c0:c0 + w].T @ z[cf.k:]
                c0 += w
            y[o:o + cf.m] = z
        stack.append(y)
        y = H._gather_next(lv, y)
    for lv in reversed([l for l in fac.levels if l.top is None]):
        yl = stack.pop()
        H._scatter_next(lv, yl, y)
        for s in reversed(lv.order):
            cf = lv.factors.get(s)
            op = None if cf is None else H.stored_operators(cf, sym)
            if op is None:
                continue
            o = lv.offsets[s]
            z = yl[o:o + cf.m].copy()
            c0 = 0
            for n, w in cf.nbrs:
                on = lv.offsets[n]
                z[cf.k:] -= op["Y"][cf.k:, c0:c0 + w] @ yl[on:on + w]
                c0 += w
            TRt = op["T"] if sym else op["TRt"]
            yl[o:o + cf.m] = TRt.T @ z
        y = yl
    x = np.empty_like(b)
    x[fac.perm] = y
    assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max()
