"""Restarted right-preconditioned GMRES(m) (Section 4: the preconditioner is
used inside GMRES; Section 6.1: iterate until the residual is reduced by
1e-6).

Textbook Arnoldi with modified Gram-Schmidt, complex Givens rotations,
zero initial guess, x = x0 + M^-1 (V y) at each restart and the true
residual ||b - A x|| / ||b|| recomputed at every restart.  The paper does not
state the Krylov details; these are the standard choices.
"""

from __future__ import annotations

import numpy as np


def givens(a: complex, b: complex):
    """(c, s, r) with [c, s; -conj(s), c] [a; b] = [r; 0], c real."""
    if b == 0:
        return 1.0, 0.0, a
    if a == 0:
        return 0.0, 1.0, b
    nu = np.hypot(abs(a), abs(b))
    ph = a / abs(a)
    return abs(a) / nu, ph * np.conj(b) / nu, ph * nu


def gmres(A, b: np.ndarray, M, m: int = 20, tol: float = 1e-6, max_iter: int = 500):
    """Solve A x = b; ``A`` and ``M`` act on flat complex vectors.

    Returns (x, info) with info = dict(iters, relres, history, converged).
    """
    b = b.ravel().astype(np.complex128)
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    hist = []
    if nb == 0:
        return x, dict(iters=0, relres=0.0, history=hist, converged=True)
    r = b.copy()
    beta = np.linalg.norm(r)
    iters = 0
    while True:
        V = np.zeros((m + 1, b.size), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        V[0] = r / beta
        g[0] = beta
        k = 0
        for j in range(m):
            w = A(M(V[j]))
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                           # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            c, s, rr = givens(H[j, j], H[j + 1, j])
            cs[j], sn[j] = c, s
            H[j, j], H[j + 1, j] = rr, 0.0
            g[j + 1] = -np.conj(s) * g[j]
            g[j] = c * g[j]
            iters += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / nb)
            if abs(g[j + 1]) / nb <= tol or iters >= max_iter:
                break
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):                   # back substitution
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + M(V[:k].T @ y)
        r = b - A(x)
        beta = np.linalg.norm(r)
        relres = beta / nb
        if relres <= tol or iters >= max_iter:
            return x, dict(iters=iters, relres=relres, history=hist, converged=relres <= tol)
