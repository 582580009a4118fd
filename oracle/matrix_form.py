"""Oracle, matrix form: Eqs. scaling, elim and perm applied as full N x N
operators to a dense matrix (tiny problems only).  Test infrastructure only.

This restates LowRank_Elimination of Alg. 1 literally: for every cluster s
the operators E_s (sparsification) and G_s (elimination) are built as N x N
matrices and applied to the whole current matrix, W A W^T, with the
approximation of Eq. lra made explicit: the fill block is replaced by U Z
before E_s is applied, after which the fine-to-far coupling vanishes.  The permutation P_s is bookkeeping of index sets.  It uses the
block oracle's clustering, colouring and compression routines (pinned on their
own) but none of its block bookkeeping, so it checks which blocks the block
oracle updates and how.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import hsolver as H


def factor_dense(A: np.ndarray, coords, leaf: int, eps: float, symmetric=True):
    """Returns dict(Winv_left, Winv_right, checks) with
    M^{-1} = R_total @ L_total where L_total = prod of left operators,
    R_total = prod of right operators (the final reduced matrix is I)."""
    n = A.shape[0]
    depth, leaves = H.rcb_leaves(np.asarray(coords, dtype=np.float64), leaf)
    Abar = np.array(A, dtype=np.float64)
    WL = np.eye(n)   # accumulated left operator
    WR = np.eye(n)   # accumulated right operator (applied as Abar @ WR^T)
    checks = dict(fine_identity=0.0, fine_decoupled=0.0, outside_d2=0.0)
    # current clusters as lists of global row indices of Abar (index space is
    # fixed: operators act in place, eliminated rows become identity rows)
    clusters = [list(map(int, x)) for x in leaves]
    eliminated = np.zeros(n, dtype=bool)
    while True:
        nclu = len(clusters)
        sizes = [len(c) for c in clusters]
        # block pattern of the current matrix restricted to live DOFs
        pairs = set()
        for i in range(nclu):
            for j in range(nclu):
                if sizes[i] and sizes[j] and np.any(Abar[np.ix_(clusters[i], clusters[j])] != 0):
                    pairs.add((i, j))
        live = sum(1 for s in sizes if s)
        if nclu == 1 or live <= 1:
            idx = [d for c in clusters for d in c]
            if idx:
                blk = Abar[np.ix_(idx, idx)]
                if symmetric:
                    L = np.linalg.cholesky(blk)
                    Linv = sla.solve_triangular(L, np.eye(len(idx)), lower=True)
                    E = np.eye(n)
                    E[np.ix_(idx, idx)] = Linv
                    Abar = E @ Abar @ E.T
                    WL = E @ WL
                    WR = E @ WR
                else:
                    P, L, U = sla.lu(blk)
                    EL = np.eye(n)
                    EL[np.ix_(idx, idx)] = sla.solve_triangular(L, P.T, lower=True, unit_diagonal=True)
                    ER = np.eye(n)
                    ER[np.ix_(idx, idx)] = sla.solve_triangular(U, np.eye(len(idx)), lower=False).T
                    Abar = EL @ Abar @ ER.T
                    WL = EL @ WL
                    WR = ER @ WR
            break
        adj = H.neighbours_from_pattern(nclu, pairs)
        d2 = H.distance2(adj)
        colour = H.greedy_colour(adj, d2)
        order = sorted(range(nclu), key=lambda i: (colour[i], i))
        coarse = [list(c) for c in clusters]
        for s in order:
            S = coarse[s]
            m = len(S)
            if m == 0:
                continue
            N = sorted(j for j in adj[s] if coarse[j])
            W = sorted(j for j in d2[s] if coarse[j])
            Widx = [d for j in W for d in coarse[j]]
            Nidx = [d for j in N for d in coarse[j]]
            # every nonzero outside s, N(s), W(s) would break Sec. 2.3
            others = [d for j in range(nclu) if j != s and j not in N and j not in W for d in coarse[j]]
            if others:
                checks["outside_d2"] = max(checks["outside_d2"],
                                           np.abs(Abar[np.ix_(S, others)]).max(initial=0.0),
                                           np.abs(Abar[np.ix_(others, S)]).max(initial=0.0))
            Ass = Abar[np.ix_(S, S)]
            G = Abar[np.ix_(S, Widx)]
            if not symmetric:
                G = np.hstack([G, Abar[np.ix_(Widx, S)].T])
            G = G[:, np.any(G != 0.0, axis=0)] if G.size else G.reshape(m, 0)
            floor = H.NOISE_FLOOR * np.abs(Ass).max()
            k = H.cpqr(G, eps, floor=floor)["k"] if G.shape[1] else 0
            if k == m:
                continue
            EL = np.eye(n)
            ER = np.eye(n)
            if k > 0:
                U = H.cpqr(G, eps, floor=floor)["U"]
                # Eq. lra: the fill block is replaced by its low-rank
                # approximation U Z, Z = U^T A_sw (and A_ws by (A_ws U) U^T)
                if Widx:
                    PU = U @ U.T
                    Abar[np.ix_(S, Widx)] = PU @ Abar[np.ix_(S, Widx)]
                    Abar[np.ix_(Widx, S)] = Abar[np.ix_(Widx, S)] @ PU
                B = np.linalg.inv(Ass)
                VL = H.complement(B @ U)
                VR = VL if symmetric else H.complement(B.T @ U)
                EL[np.ix_(S, S)] = np.vstack([U.T, VL.T]) @ B
                ER[np.ix_(S, S)] = np.vstack([U.T, VR.T]) @ B.T
            Abar = EL @ Abar @ ER.T
            WL = EL @ WL
            WR = ER @ WR
            fine = S[k:]
            crs = S[:k]
            if crs:
                checks["fine_decoupled"] = max(checks["fine_decoupled"],
                                               np.abs(Abar[np.ix_(fine, crs)]).max(),
                                               np.abs(Abar[np.ix_(crs, fine)]).max())
            # with the fill block replaced, the fine-to-far coupling vanishes
            if Widx:
                checks["fine_far"] = max(checks.get("fine_far", 0.0),
                                         np.abs(Abar[np.ix_(fine, Widx)]).max(initial=0.0),
                                         np.abs(Abar[np.ix_(Widx, fine)]).max(initial=0.0))
                Abar[np.ix_(fine, Widx)] = 0.0
                Abar[np.ix_(Widx, fine)] = 0.0
            # Eq. elim: G_s with the factor of the fine block
            F = Abar[np.ix_(fine, fine)]
            GL = np.eye(n)
            GR = np.eye(n)
            rest = [d for d in range(n) if d not in set(fine) and not eliminated[d]]
            if symmetric:
                L = np.linalg.cholesky(F)
                Linv = sla.solve_triangular(L, np.eye(len(fine)), lower=True)
                GL[np.ix_(fine, fine)] = Linv
                GR[np.ix_(fine, fine)] = Linv
            else:
                P, L, U = sla.lu(F)
                GL[np.ix_(fine, fine)] = sla.solve_triangular(L, P.T, lower=True, unit_diagonal=True)
                GR[np.ix_(fine, fine)] = sla.solve_triangular(U, np.eye(len(fine)), lower=False).T
            Abar = GL @ Abar @ GR.T
            WL = GL @ WL
            WR = GR @ WR
            # second factor of G_s: clear the fine columns/rows of the rest
            GL2 = np.eye(n)
            GR2 = np.eye(n)
            GL2[np.ix_(rest, fine)] = -Abar[np.ix_(rest, fine)]
            GR2[np.ix_(rest, fine)] = -Abar[np.ix_(fine, rest)].T
            Abar = GL2 @ Abar @ GR2.T
            WL = GL2 @ WL
            WR = GR2 @ WR
            checks["fine_identity"] = max(checks["fine_identity"],
                                          np.abs(Abar[np.ix_(fine, fine)] - np.eye(len(fine))).max())
            eliminated[fine] = True
            coarse[s] = crs
        clusters = [coarse[2 * I] + coarse[2 * I + 1] for I in range(nclu // 2)]
    # Abar is now (numerically) the identity: A ~= WL^{-1} WR^{-T}
    Minv = WR.T @ WL
    checks["final_identity"] = np.abs(Abar - np.eye(n)).max()
    return dict(Minv=Minv, checks=checks)
