"""Oracle: the hierarchical factorization (Alg. 1) and solve (Alg. 2), float64.

Test infrastructure only -- never imported by the library.

Notation follows Sec. 2 of the paper: a level's matrix is partitioned into
clusters pi_i; when cluster s is processed, n are its neighbours in the block
pattern A_B of the level (Eq. quotient), w the clusters at block distance
exactly two (the only place fill-in can live, Sec. 2.3).  The fill block
A_sw is compressed (Eq. lra) to an orthonormal basis U, an orthonormal V with
V^T A_ss^{-1} U = 0 is built, the sparsification operator E_s (Eq. scaling)
splits pi_s into fine and coarse DOFs, the elimination operator G_s (Eq.
elim) removes the fine ones, and P_s (Eq. perm) leaves the coarse ones to the
next level, where siblings of the bisection tree merge (Alg. 1, recursion).

Readings of points the paper leaves open:
  * Clustering: recursive coordinate bisection to a uniform depth; each node
    is split at the median of its longest bounding-box axis (ties: lowest
    axis), ordering points by (coordinate, global index); the left half gets
    floor(size/2).  Level-l clusters are the nodes l levels above the leaves;
    a level-(l+1) cluster holds the coarse DOFs of its two children, left
    child first.
  * Order: greedy distance-2 colouring of A_B in smallest-last order (the
    cluster with the fewest remaining distance-<=2 neighbours removed first,
    ties to the lowest index, colours given in reverse removal order);
    clusters are processed by (colour, index).  Clusters of one colour are >2 apart
    (Sec. 3.2), so their order does not change any value.
  * Fill basis: Householder QR with column pivoting of G = [A_sw] (symmetric)
    or [A_sw, A_ws^T] (general), w in increasing order; column norms are
    recomputed at every step; the pivot is the column of largest remaining
    norm, near-ties (squared norm within a relative 1e-10 of the largest)
    going to the lowest original column index; the factorization stops at the
    first step j with |r_jj| <= eps |r_11| (eps > 0), with |r_jj| <=
    1e-14 max|A_ss| (a fill block at the rounding level of the cluster's own
    diagonal block is zero in exact arithmetic; without this floor its
    "rank" is decided by rounding noise), or when the remaining columns are
    all exactly zero.  k = number of kept steps, U = first k columns of Q.
  * Randomized variant (a randomized rank-revealing QR): when
    G has more than m + 8 columns, the same truncated pivoted QR runs on the
    sketch G Omega with Omega[q, j] = +-1/sqrt(m + 8), signs from the top
    bit of splitmix64((q << 32) | j), q the gathered column position.  With
    m + 8 >= m columns the sketch spans the column space of G exactly (with
    probability one), so eps = 0 stays a direct solver.
  * k = 0 (no fill): E_s = I and the step is one block-Cholesky/LU step
    (Sec. 2.2).  k = m: the cluster is left untouched (E_s = I, all coarse).
  * Householder convention: v = x - beta e1, beta = -sign(x_0) ||x||
    (sign(0) = +1), H = I - 2 v v^T / v^T v.  The compression basis U is
    then oriented so that R has a positive diagonal (column j of Q times
    sign(beta_j)), i.e. U's columns are the Gram-Schmidt directions of the
    pivot columns.  The sign of beta follows the sign of x_0, which rounding
    decides when x_0 is near zero; with this orientation the coarse bases,
    and every coarse block built from them, are continuous functions of the
    data (the randomized variant below depends on those signs).
    The complement V keeps the plain Householder columns: its basis only
    touches the eliminated fine unknowns.
  * General (nonsymmetric) matrices: one joint basis U for the row and column
    fill; V_L is the complement of A_ss^{-1} U and V_R that of A_ss^{-T} U, so
    that the coarse/fine (s,s) coupling vanishes on both sides; the fine block
    F = V_L^T A_ss^{-1} V_R is factored by LU with partial pivoting.
  * Coarse-to-far coupling: (U^T A_ss^{-1} U) Z with Z = U^T A_sw (Eq. scaling's
    display); fine-to-far coupling is dropped.
  * Next level's A_B: block (I, J) is present iff some child pair (a, b) was
    within block distance two at this level and both kept coarse DOFs.
  * Top: when one cluster is left, or the level holds at most ``top_size``
    DOFs, the whole level is factored densely (Alg. 1, "small enough": a size
    test, the same for SPD and general matrices): Cholesky, or LU with
    partial pivoting for a general matrix (Sec. 6).
  * Alg. 2's backward sweep: the coarse system is solved before W_i^T is
    applied for i = m-1..0 -- the order that inverts the factorization of
    Alg. 1 (A^fac = W_0^{-1} .. W_{m-1}^{-1} diag(I, A_c^fac) W_{m-1}^{-T} ..).
"""
from __future__ import annotations

import dataclasses
import numpy as np
import scipy.linalg as sla

PIVOT_TIE_RTOL = 1e-10
# A fill direction whose |r_jj| is at most this fraction of max |A_ss| is
# rounding noise of a block that is zero in exact arithmetic; it is dropped
# whatever eps is (see the module docstring).
NOISE_FLOOR = 1e-14


# ---------------------------------------------------------------------------
# Clustering (Alg. 1, partition step)
# ---------------------------------------------------------------------------

def rcb_leaves(coords: np.ndarray, leaf: int):
    """Recursive coordinate bisection to a uniform depth.

    Returns (depth, leaves) where leaves is a list of 2**depth int64 arrays of
    global DOF indices (each sorted ascending), in left-to-right tree order.
    """
    n = coords.shape[0]
    depth = 0
    while -(-n // (1 << depth)) > leaf:
        depth += 1
    nodes = [np.arange(n, dtype=np.int64)]
    for _ in range(depth):
        nxt = []
        for idx in nodes:
            if len(idx) == 0:
                nxt += [idx, idx]
                continue
            c = coords[idx]
            ext = c.max(axis=0) - c.min(axis=0)
            ax = int(np.argmax(ext))  # first maximum: lowest axis on ties
            order = np.lexsort((idx, c[:, ax]))
            half = len(idx) // 2
            nxt.append(idx[order[:half]])
            nxt.append(idx[order[half:]])
        nodes = nxt
    return depth, [np.sort(x) for x in nodes]


# ---------------------------------------------------------------------------
# Block pattern and colouring (Eq. quotient, Sec. 2.3, Sec. 3.2)
# ---------------------------------------------------------------------------

def neighbours_from_pattern(nclu: int, pairs):
    """Adjacency sets (excluding self) from an iterable of (i, j) block ids."""
    adj = [set() for _ in range(nclu)]
    for i, j in pairs:
        if i != j:
            adj[i].add(j)
            adj[j].add(i)
    return adj


def distance2(adj):
    """For every cluster, the clusters at block distance exactly two."""
    out = []
    for i, nb in enumerate(adj):
        d2 = set()
        for j in nb:
            d2 |= adj[j]
        d2 -= nb
        d2.discard(i)
        out.append(d2)
    return out


def smallest_last_order(adj, d2):
    """Smallest-last vertex order of the distance-<=2 graph: repeatedly
    remove the remaining cluster with the fewest remaining distance-<=2
    neighbours (ties: lowest index); the order is the reverse of the
    removals."""
    import heapq
    nb = [adj[i] | d2[i] for i in range(len(adj))]
    deg = [len(x) for x in nb]
    heap = [(deg[i], i) for i in range(len(adj))]
    heapq.heapify(heap)
    removed = [False] * len(adj)
    order = []
    while heap:
        d, i = heapq.heappop(heap)
        if removed[i] or d != deg[i]:
            continue  # a stale entry
        removed[i] = True
        order.append(i)
        for j in nb[i]:
            if not removed[j]:
                deg[j] -= 1
                heapq.heappush(heap, (deg[j], j))
    return order[::-1]


def greedy_colour(adj, d2):
    """Greedy distance-2 colouring (smallest free colour) in smallest-last
    order.  The paper asks its colouring for few colours (Sec. 3.4); this
    order gives fewer classes than index order on the coarse levels."""
    col = [-1] * len(adj)
    for i in smallest_last_order(adj, d2):
        used = {col[j] for j in (adj[i] | d2[i]) if col[j] >= 0}
        c = 0
        while c in used:
            c += 1
        col[i] = c
    return col


# ---------------------------------------------------------------------------
# Sketch for the randomized variant of Eq. lra
# ---------------------------------------------------------------------------

SKETCH_OVERSAMPLE = 8
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x):
    """SplitMix64 output function (Steele, Lea, Flood 2014; Vigna's public
    domain reference): one 64-bit output per 64-bit input, uint64 arrays."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def sketch_matrix(c: int, l: int) -> np.ndarray:
    """Rademacher test matrix Omega (c x l): Omega[q, j] = +-1/sqrt(l), the
    sign being the top bit of splitmix64((q << 32) | j)."""
    q = np.arange(c, dtype=np.uint64)[:, None]
    j = np.arange(l, dtype=np.uint64)[None, :]
    z = splitmix64((q << np.uint64(32)) | j)
    return (1.0 - 2.0 * (z >> np.uint64(63)).astype(np.float64)) / np.sqrt(l)


# ---------------------------------------------------------------------------
# Householder pieces (shared convention, see module docstring)
# ---------------------------------------------------------------------------

def householder(x: np.ndarray):
    """Return (v, tau, beta) with (I - tau v v^T) x = beta e1."""
    x = np.asarray(x, dtype=np.float64)
    nrm = np.sqrt(np.dot(x, x))
    if nrm == 0.0:
        return np.zeros_like(x), 0.0, 0.0
    beta = -nrm if x[0] >= 0 else nrm
    v = x.copy()
    v[0] -= beta
    tau = 2.0 / np.dot(v, v)
    return v, tau, beta


def cpqr(G: np.ndarray, eps: float, max_rank: int | None = None, floor: float = 0.0):
    """Householder QR with column pivoting, truncated at eps (Eq. lra).

    The factorization stops at the first step whose |r_jj| is at or below
    eps |r_11| (eps > 0) or at or below the absolute `floor`.  Returns
    dict(k, U, piv, rdiag, margin) where U (m x k) has orthonormal columns
    spanning the kept directions, piv are the chosen original column indices
    and rdiag the |r_jj| of every kept step.
    """
    m, c = G.shape
    A = np.array(G, dtype=np.float64, copy=True)
    cols = np.arange(c)
    vs, taus, piv, rdiag, signs = [], [], [], [], []
    r11 = None
    k = 0
    margin = np.inf
    kmax = min(m, c) if max_rank is None else min(m, c, max_rank)
    for j in range(min(m, c)):
        sub = A[j:, j:]
        nrm2 = np.einsum("ij,ij->j", sub, sub)
        mx = nrm2.max()
        if mx == 0.0:
            break
        cand = np.nonzero(nrm2 >= (1.0 - PIVOT_TIE_RTOL) * mx)[0]
        p = cand[np.argmin(cols[j + cand])]
        r = np.sqrt(nrm2[p])
        if j == 0:
            r11 = r
        if r <= floor:
            break
        if eps > 0.0:
            margin = min(margin, abs(r / (eps * r11) - 1.0))
            if r <= eps * r11:
                break
        if j >= kmax:
            break
        # swap pivot column into position j
        q = j + p
        A[:, [j, q]] = A[:, [q, j]]
        cols[[j, q]] = cols[[q, j]]
        v, tau, beta = householder(A[j:, j])
        A[j:, j:] -= tau * np.outer(v, v @ A[j:, j:])
        vs.append(v)
        taus.append(tau)
        signs.append(-1.0 if beta < 0 else 1.0)
        piv.append(int(cols[j]))
        rdiag.append(float(r))
        k = j + 1
    # U = H_0 ... H_{k-1} [I_k; 0], each column j then signed like beta_j so
    # that R has a positive diagonal (see the module docstring)
    U = np.zeros((m, k))
    U[:k, :k] = np.eye(k)
    for j in range(k - 1, -1, -1):
        v, tau = vs[j], taus[j]
        U[j:, :] -= tau * np.outer(v, v @ U[j:, :])
    U *= np.array(signs[:k]) if k else 1.0
    return dict(k=k, U=U, piv=piv, rdiag=rdiag, margin=margin)


def complement(X: np.ndarray):
    """Orthonormal V (m x (m-k)) with V^T X = 0, from the full Householder QR
    of X (no pivoting): V = Q[:, k:]."""
    m, k = X.shape
    A = np.array(X, dtype=np.float64, copy=True)
    vs, taus = [], []
    for j in range(k):
        v, tau, _ = householder(A[j:, j])
        A[j:, j:] -= tau * np.outer(v, v @ A[j:, j:])
        vs.append(v)
        taus.append(tau)
    V = np.zeros((m, m - k))
    V[k:, :] = np.eye(m - k)
    for j in range(k - 1, -1, -1):
        v, tau = vs[j], taus[j]
        V[j:, :] -= tau * np.outer(v, v @ V[j:, :])
    return V


# ---------------------------------------------------------------------------
# Factor records
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class ClusterFactor:
    s: int
    m: int            # DOFs of s when processed
    k: int            # coarse DOFs kept
    TL: np.ndarray | None   # m x m, rows [U^T; V_L^T] A_ss^{-1}  (None: identity)
    TR: np.ndarray | None   # m x m, A_ss^{-1} [U, V_R]          (None: identity)
    LF: np.ndarray          # f x f lower factor of F (unit-lower if LU)
    UF: np.ndarray          # f x f upper factor of F (= LF^T if Cholesky)
    PF: np.ndarray          # f permutation of F's rows (identity if Cholesky)
    nbrs: list              # [(n, width)] neighbour slots touched
    BL: np.ndarray          # (sum width) x f : C_nf U_F^{-1}
    BR: np.ndarray          # f x (sum width) : L_F^{-1} P_F R_fn
    piv: list
    rdiag: list
    margin: float
    ncols_fill: int         # nonzero columns of G
    # recorded for comparisons with other implementations (no later step
    # reads them): A_ss as the cluster met it, its new coarse rows
    # U^T A_ss^{-1} A_sN (k x sum width) and coarse columns A_Ns A_ss^{-1} U
    Ass: np.ndarray | None = None
    Yc: np.ndarray | None = None
    Xc: np.ndarray | None = None


@dataclasses.dataclass
class Level:
    nclu: int
    sizes: np.ndarray       # DOFs per cluster at level start
    offsets: np.ndarray     # slot offsets in the level vector
    adj: list
    d2: list
    colour: list
    order: list
    factors: dict           # s -> ClusterFactor
    ranks: np.ndarray       # coarse DOFs per cluster after the level
    top: dict | None = None  # dense top factor (if this level is the top)


@dataclasses.dataclass
class Factorization:
    n: int
    symmetric: bool
    perm: np.ndarray        # level-0 vector position -> global DOF
    levels: list


# ---------------------------------------------------------------------------
# Factorization (Alg. 1)
# ---------------------------------------------------------------------------

def _level0_blocks(rowptr, col, val, leaves):
    n = len(rowptr) - 1
    clu = np.empty(n, dtype=np.int64)
    loc = np.empty(n, dtype=np.int64)
    for i, idx in enumerate(leaves):
        clu[idx] = i
        loc[idx] = np.arange(len(idx))
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    ci, cj = clu[rows], clu[col]
    pairs = set(zip(ci.tolist(), cj.tolist()))
    sizes = np.array([len(x) for x in leaves])
    blocks = {}
    for (i, j) in pairs:
        blocks[(i, j)] = np.zeros((sizes[i], sizes[j]))
    for r, c, v, a, b in zip(rows.tolist(), col.tolist(), val.tolist(), ci.tolist(), cj.tolist()):
        blocks[(a, b)][loc[r], loc[c]] += v
    return sizes, pairs, blocks


def _dense_top(blocks, sizes, symmetric):
    offs = np.concatenate([[0], np.cumsum(sizes)])
    n = int(offs[-1])
    A = np.zeros((n, n))
    for (i, j), b in blocks.items():
        if sizes[i] and sizes[j]:
            A[offs[i]:offs[i + 1], offs[j]:offs[j + 1]] = b[:sizes[i], :sizes[j]]
    if n == 0:
        return dict(n=0, kind="empty")
    if symmetric:
        try:
            L = np.linalg.cholesky(A)
        except np.linalg.LinAlgError as e:
            raise np.linalg.LinAlgError("top block not SPD") from e
        return dict(n=n, kind="chol", L=L)
    P, L, U = sla.lu(A)
    return dict(n=n, kind="lu", P=P, L=L, U=U)


def _process_cluster(s, blocks, cur, adj, d2, eps, symmetric, max_rank, compress=0):
    m = cur[s]
    N = sorted(j for j in adj[s] if cur[j] > 0)
    W = sorted(j for j in d2[s] if cur[j] > 0 and (s, j) in blocks)
    Ass = blocks[(s, s)][:m, :m]
    # --- Eq. lra: compress the fill blocks
    parts = [blocks[(s, w)][:m, :cur[w]] for w in W]
    if not symmetric:
        parts += [blocks[(w, s)][:cur[w], :m].T for w in W]
    G = np.hstack(parts) if parts else np.zeros((m, 0))
    floor = NOISE_FLOOR * np.abs(Ass).max()
    l = m + SKETCH_OVERSAMPLE
    if compress == 1 and G.shape[1] > l:
        # randomized variant: the same pivoted QR on the sketch G Omega,
        # Omega indexed by the gathered column position (zero columns too)
        cp = cpqr(G @ sketch_matrix(G.shape[1], l), eps, max_rank, floor=floor)
        G = G[:, np.any(G != 0.0, axis=0)]
    else:
        G = G[:, np.any(G != 0.0, axis=0)]
        if G.shape[1] == 0:
            cp = dict(k=0, U=np.zeros((m, 0)), piv=[], rdiag=[], margin=np.inf)
        else:
            cp = cpqr(G, eps, max_rank, floor=floor)
    k = cp["k"]
    widths = [(n, cur[n]) for n in N]
    AsN = np.hstack([blocks[(s, n)][:m, :w] for n, w in widths]) if N else np.zeros((m, 0))
    ANs = np.vstack([blocks[(n, s)][:w, :m] for n, w in widths]) if N else np.zeros((0, m))
    Ass0 = Ass.copy()
    if k == m:
        # untouched: all DOFs coarse, E_s = I
        return ClusterFactor(s, m, m, None, None, np.zeros((0, 0)), np.zeros((0, 0)),
                             np.zeros(0, dtype=np.int64), widths, np.zeros((AsN.shape[1], 0)),
                             np.zeros((0, AsN.shape[1])), cp["piv"], cp["rdiag"], cp["margin"],
                             G.shape[1], Ass0)
    if k == 0:
        # no fill kept: E_s = I, plain block elimination (Sec. 2.2)
        TL = TR = None
        F = Ass.copy()
        R = AsN
        Cn = ANs
        Yc = np.zeros((0, AsN.shape[1]))
        Xc = np.zeros((ANs.shape[0], 0))
    else:
        U = cp["U"]
        B = np.linalg.solve(Ass, np.eye(m))          # A_ss^{-1}
        VL = complement(B @ U)                        # V_L^T A_ss^{-1} U = 0
        VR = VL if symmetric else complement(B.T @ U)  # U^T A_ss^{-1} V_R = 0
        TL = np.vstack([U.T @ B, VL.T @ B])           # E_s restricted to s
        TR = TL.T if symmetric else np.hstack([B @ U, B @ VR])  # E_s^T (right side)
        C = U.T @ B @ U                               # coarse (s,s) block
        F = VL.T @ B @ VR                             # fine (s,s) block
        Y = TL @ AsN                                  # [U^T B A_sN; V_L^T B A_sN]
        X = Y.T if symmetric else ANs @ TR            # [A_Ns B U, A_Ns B V_R]
        R = Y[k:]
        Cn = X[:, k:]
        Yc = Y[:k].copy()
        Xc = X[:, :k].copy()
        # new coarse rows/cols of s (Eq. scaling, display)
        col0 = 0
        for n, w in widths:
            blocks[(s, n)][:k, :w] = Y[:k, col0:col0 + w]
            blocks[(n, s)][:w, :k] = X[col0:col0 + w, :k]
            col0 += w
        for w_ in W:
            cw = cur[w_]
            Z = U.T @ blocks[(s, w_)][:m, :cw]
            Zt = blocks[(w_, s)][:cw, :m] @ U
            blocks[(s, w_)][:k, :cw] = C @ Z
            blocks[(w_, s)][:cw, :k] = Zt @ C
        blocks[(s, s)][:k, :k] = C
    f = m - k
    # --- Eq. elim: factor the fine block and form the Schur update
    if symmetric:
        try:
            LF = np.linalg.cholesky(F)
        except np.linalg.LinAlgError as e:
            raise np.linalg.LinAlgError(f"fine block of cluster {s} not SPD") from e
        UF = LF.T
        PF = np.arange(f)
    else:
        P, LF, UF = sla.lu(F)
        PF = np.argmax(P, axis=0)  # row i of P^T F comes from row PF[i]
    BR = sla.solve_triangular(LF, R[PF], lower=True, unit_diagonal=not symmetric) if f else np.zeros((0, R.shape[1]))
    BL = sla.solve_triangular(UF.T, Cn.T, lower=True).T if f else np.zeros((Cn.shape[0], 0))
    # Schur complement on the neighbour blocks: A_NN -= B_L B_R
    r0 = 0
    for n1, w1 in widths:
        c0 = 0
        for n2, w2 in widths:
            blocks[(n1, n2)][:w1, :w2] -= BL[r0:r0 + w1] @ BR[:, c0:c0 + w2]
            c0 += w2
        r0 += w1
    return ClusterFactor(s, m, k, TL, TR, LF, UF, PF, widths, BL, BR, cp["piv"], cp["rdiag"],
                         cp["margin"], G.shape[1], Ass0, Yc, Xc)


def factor(prob_rowptr, prob_col, prob_val, coords, leaf: int, eps: float,
           symmetric: bool = True, top_size: int = 0, max_rank: int | None = None,
           compress: int = 0):
    """Hierarchical_Factor (Alg. 1) on a CSR matrix.  Returns a Factorization.

    compress = 0: pivoted QR of the fill block G itself (Eq. lra);
    compress = 1: when G has more than m + 8 columns, pivoted QR of the
    sketch G Omega (m x (m + 8), Rademacher Omega from `sketch_matrix`)
    instead -- the randomized rank-revealing variant."""
    depth, leaves = rcb_leaves(np.asarray(coords, dtype=np.float64), leaf)
    perm = np.concatenate(leaves).astype(np.int64)
    sizes, pairs, blocks = _level0_blocks(prob_rowptr, prob_col, prob_val, leaves)
    nclu = len(leaves)
    adj = neighbours_from_pattern(nclu, pairs)
    levels = []
    while True:
        sizes = np.asarray(sizes, dtype=np.int64)
        offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        d2 = distance2(adj)
        live = int(np.count_nonzero(sizes))
        if nclu == 1 or live <= 1 or offsets[-1] <= top_size:
            top = _dense_top(blocks, sizes, symmetric)
            levels.append(Level(nclu, sizes, offsets, adj, d2, [0] * nclu, list(range(nclu)), {},
                                np.zeros(nclu, dtype=np.int64), top))
            break
        # storage for every block within distance two (fill lands there)
        for i in range(nclu):
            for j in adj[i] | d2[i]:
                if (i, j) not in blocks:
                    blocks[(i, j)] = np.zeros((sizes[i], sizes[j]))
        colour = greedy_colour(adj, d2)
        order = sorted(range(nclu), key=lambda i: (colour[i], i))
        cur = sizes.copy()
        facs = {}
        for s in order:
            if cur[s] == 0:
                continue
            cf = _process_cluster(s, blocks, cur, adj, d2, eps, symmetric, max_rank, compress)
            facs[s] = cf
            cur[s] = cf.k
        levels.append(Level(nclu, sizes, offsets, adj, d2, colour, order, facs, cur.copy()))
        # --- merge siblings: coarse DOFs of children 2I, 2I+1 (left first)
        nxt = nclu // 2
        nsizes = np.array([cur[2 * I] + cur[2 * I + 1] for I in range(nxt)], dtype=np.int64)
        nblocks = {}
        npairs = set()
        for (a, b), blk in blocks.items():
            if cur[a] == 0 or cur[b] == 0:
                continue
            I, J = a // 2, b // 2
            if (I, J) not in nblocks:
                nblocks[(I, J)] = np.zeros((nsizes[I], nsizes[J]))
            ro = 0 if a % 2 == 0 else cur[a - 1]
            co = 0 if b % 2 == 0 else cur[b - 1]
            nblocks[(I, J)][ro:ro + cur[a], co:co + cur[b]] = blk[:cur[a], :cur[b]]
            npairs.add((I, J))
        blocks = nblocks
        adj = neighbours_from_pattern(nxt, npairs)
        sizes = nsizes
        nclu = nxt
    return Factorization(len(prob_rowptr) - 1, symmetric, perm, levels)


def stored_operators(cf: ClusterFactor, symmetric: bool):
    """The operators of one processed cluster in the form an implementation
    that folds the fine block's factors into the sparsification rows stores
    them (Eqs. scaling and elim combined):

      T   = [U^T A_ss^{-1}; L_F^{-1} P_F V_L^T A_ss^{-1}]       (m x m)
      TRt = [U^T A_ss^{-T}; U_F^{-T} V_R^T A_ss^{-T}]           (general)
      Y   = [U^T A_ss^{-1} A_sN; B_R]                          (m x sum width)
      XT  = [(A_Ns A_ss^{-1} U)^T; B_L^T]                      (general)

    With k = 0 (E_s = I) the sparsification rows are the identity: T =
    L_F^{-1} P_F and TRt = U_F^{-T} for F = A_ss.  A cluster with k = m keeps
    no operators (returns None)."""
    m, k = cf.m, cf.k
    if k == m:
        return None
    f = m - k
    unit = not symmetric
    if cf.TL is None:
        TL = np.eye(m)
        TRm = np.eye(m)
    else:
        TL = cf.TL
        TRm = cf.TL.T if symmetric else cf.TR
    T = np.vstack([TL[:k], sla.solve_triangular(cf.LF, TL[k:][cf.PF], lower=True,
                                                 unit_diagonal=unit)])
    Y = np.vstack([cf.Yc, cf.BR])
    out = dict(T=T, Y=Y, TRt=None, XT=None)
    if not symmetric:
        out["TRt"] = np.vstack([TRm[:, :k].T,
                                sla.solve_triangular(cf.UF.T, TRm[:, k:].T, lower=True)])
        out["XT"] = np.vstack([cf.Xc.T, cf.BL.T])
    assert T.shape == (m, m) and Y.shape[0] == m and cf.BR.shape[0] == f
    return out


def top_operators(top: dict):
    """The dense top in the same form: T = L^{-1} (Cholesky A = L L^T) or,
    for an LU top A = P L U, T = L^{-1} P^T and TRt = U^{-T}.  An empty top
    (no unknown left) has none (returns None)."""
    n = top["n"]
    if n == 0:
        return None
    if top["kind"] == "chol":
        return dict(T=sla.solve_triangular(top["L"], np.eye(n), lower=True), TRt=None)
    T = sla.solve_triangular(top["L"], top["P"].T, lower=True, unit_diagonal=True)
    return dict(T=T, TRt=sla.solve_triangular(top["U"].T, np.eye(n), lower=True))


# ---------------------------------------------------------------------------
# Solve (Alg. 2)
# ---------------------------------------------------------------------------

def _forward_cluster(cf: ClusterFactor, y, offsets, symmetric):
    o = offsets[cf.s]
    ys = y[o:o + cf.m]
    if cf.k == cf.m:
        return
    if cf.TL is not None:
        ys[:] = cf.TL @ ys
    k = cf.k
    yf = ys[k:]
    yf[:] = sla.solve_triangular(cf.LF, yf[cf.PF], lower=True, unit_diagonal=not symmetric)
    r0 = 0
    for n, w in cf.nbrs:
        on = offsets[n]
        y[on:on + w] -= cf.BL[r0:r0 + w] @ yf
        r0 += w


def _backward_cluster(cf: ClusterFactor, x, offsets):
    o = offsets[cf.s]
    xs = x[o:o + cf.m]
    if cf.k == cf.m:
        return
    k = cf.k
    xf = xs[k:].copy()
    c0 = 0
    for n, w in cf.nbrs:
        on = offsets[n]
        xf -= cf.BR[:, c0:c0 + w] @ x[on:on + w]
        c0 += w
    xs[k:] = sla.solve_triangular(cf.UF, xf, lower=False)
    if cf.TR is not None:
        xs[:] = cf.TR @ xs


def _gather_next(lv: Level, y):
    parts = []
    for I in range(lv.nclu // 2):
        for a in (2 * I, 2 * I + 1):
            o = lv.offsets[a]
            parts.append(y[o:o + lv.ranks[a]])
    return np.concatenate(parts) if parts else np.zeros((0,) + y.shape[1:])


def _scatter_next(lv: Level, y, yc):
    p = 0
    for I in range(lv.nclu // 2):
        for a in (2 * I, 2 * I + 1):
            o = lv.offsets[a]
            r = lv.ranks[a]
            y[o:o + r] = yc[p:p + r]
            p += r


def solve(fac: Factorization, b: np.ndarray) -> np.ndarray:
    """x = M^{-1} b, M = A^fac (Alg. 2).  b has shape (n,) or (n, nrhs)."""
    b = np.asarray(b, dtype=np.float64)
    vec = b.ndim == 1
    bb = b[:, None] if vec else b
    y = bb[fac.perm].copy()
    stack = []
    for lv in fac.levels:
        if lv.top is not None:
            t = lv.top
            if t["kind"] == "chol":
                z = sla.solve_triangular(t["L"], y, lower=True)
                y = sla.solve_triangular(t["L"].T, z, lower=False)
            elif t["kind"] == "lu":
                z = sla.solve_triangular(t["L"], t["P"].T @ y, lower=True, unit_diagonal=True)
                y = sla.solve_triangular(t["U"], z, lower=False)
            break
        for s in lv.order:
            if s in lv.factors:
                _forward_cluster(lv.factors[s], y, lv.offsets, fac.symmetric)
        stack.append(y)
        y = _gather_next(lv, y)
    # backward: coarse first, then W_i^T for i = m-1 .. 0
    for lv in reversed([l for l in fac.levels if l.top is None]):
        yl = stack.pop()
        _scatter_next(lv, yl, y)
        for s in reversed(lv.order):
            if s in lv.factors:
                _backward_cluster(lv.factors[s], yl, lv.offsets)
        y = yl
    x = np.empty_like(bb)
    x[fac.perm] = y
    return x[:, 0] if vec else x


def stats(fac: Factorization):
    """Per-level summary: clusters, colours, DOFs in/out, rank histogram."""
    out = []
    for li, lv in enumerate(fac.levels):
        if lv.top is not None:
            out.append(dict(level=li, top=lv.top["n"], nclu=lv.nclu))
            continue
        ks = [f.k for f in lv.factors.values()]
        out.append(dict(level=li, nclu=lv.nclu, colours=max(lv.colour) + 1,
                        dofs=int(lv.offsets[-1]), coarse=int(lv.ranks.sum()),
                        mmax=int(lv.sizes.max()), kmax=max(ks) if ks else 0,
                        kmean=float(np.mean(ks)) if ks else 0.0,
                        fillcols_max=max((f.ncols_fill for f in lv.factors.values()), default=0),
                        nbr_width_max=max((sum(w for _, w in f.nbrs) for f in lv.factors.values()), default=0)))
    return out
