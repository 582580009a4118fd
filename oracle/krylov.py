"""Oracle: Krylov solvers with the hierarchical factorization as preconditioner
(Sec. 5: CG for SPD systems, GMRES otherwise).  Test infrastructure only.

Both start from x = 0 and stop when ||b - A x||_2 <= tol ||b||_2 for the
right-hand side (one at a time; the relative residual is recomputed from
scratch, b - A x, when the recurrence says it has converged).
"""
from __future__ import annotations

import numpy as np


def pcg(A, b, precond, tol=1e-10, maxit=1000):
    """Preconditioned conjugate gradients (Hestenes-Stiefel form).

    A: callable or matrix with @; precond: callable r -> M^{-1} r.
    Returns (x, iterations, relative residual)."""
    mv = A if callable(A) else (lambda v: A @ v)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    if nb == 0.0:
        return x, 0, 0.0
    r = b.copy()
    z = precond(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = mv(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        if np.linalg.norm(r) <= tol * nb:
            true = np.linalg.norm(b - mv(x)) / nb
            if true <= tol:
                return x, it, true
        z = precond(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, np.linalg.norm(b - mv(x)) / nb


def fgmres(A, b, precond, tol=1e-10, maxit=1000, restart=50):
    """Right-preconditioned flexible GMRES(restart), classical Gram-Schmidt
    applied twice (CGS2), Givens rotations for the least-squares problem.
    Returns (x, iterations, relative residual)."""
    mv = A if callable(A) else (lambda v: A @ v)
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    if nb == 0.0:
        return x, 0, 0.0
    total = 0
    while total < maxit:
        r = b - mv(x)
        beta = np.linalg.norm(r)
        if beta <= tol * nb:
            return x, total, beta / nb
        V = np.zeros((n, restart + 1))
        Z = np.zeros((n, restart))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[:, 0] = r / beta
        j_done = 0
        for j in range(restart):
            Z[:, j] = precond(V[:, j])
            w = mv(Z[:, j])
            h = V[:, :j + 1].T @ w
            w = w - V[:, :j + 1] @ h
            h2 = V[:, :j + 1].T @ w
            w = w - V[:, :j + 1] @ h2
            h = h + h2
            H[:j + 1, j] = h
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[:, j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            j_done = j + 1
            if abs(g[j + 1]) <= tol * nb or total >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + Z[:, :j_done] @ y
        res = np.linalg.norm(b - mv(x))
        if res <= tol * nb:
            return x, total, res / nb
    return x, total, np.linalg.norm(b - mv(x)) / nb
