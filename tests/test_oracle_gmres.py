"""Pins of the oracle's GMRES(m) (oracle/gmres.py; the Krylov solver the
preconditioner serves, Section 4 and Section 6.1).

GMRES is defined by a minimisation: the k-th iterate of a cycle started at
x0 = 0 minimises ||b - A M z|| over the Krylov space
K_k = span{b, (A M) b, ..., (A M)^(k-1) b}, and x = M z.  The tests compute
that minimum independently, by a dense least-squares problem over an
explicitly built Krylov basis, and compare it with the residual history the
oracle reports.  They also check finite termination on a diagonalisable
matrix with few distinct eigenvalues, and the restart bookkeeping.  A
plausible mistake planted in its source (a rotation without the conjugate, a
Gram-Schmidt coefficient without the conjugate, earlier rotations skipped)
fails the minimisation pin.
"""

from __future__ import annotations

import inspect
import textwrap

import numpy as np
import pytest

from oracle import gmres as G

N = 12


def _system(seed):
    rng = np.random.default_rng(seed)
    A = np.eye(N) * (3.0 + 1.0j) + 0.4 * (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)))
    Mm = np.eye(N) + 0.1 * (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)))
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    return A, Mm, b


def _min_residuals(A, Mm, b, kmax):
    """min_{z in K_k} ||b - A M z|| / ||b|| for k = 1..kmax, by least squares
    over an orthonormalised Krylov basis."""
    AM = A @ Mm
    K = [b]
    for _ in range(kmax - 1):
        K.append(AM @ K[-1])
    out = []
    for k in range(1, kmax + 1):
        Q, _ = np.linalg.qr(np.stack(K[:k], axis=1))
        z, *_ = np.linalg.lstsq(AM @ Q, b, rcond=None)
        out.append(np.linalg.norm(b - AM @ Q @ z) / np.linalg.norm(b))
    return np.array(out)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_residual_history_is_the_krylov_minimum(seed):
    A, Mm, b = _system(seed)
    kmax = 6
    x, info = G.gmres(lambda v: A @ v, b, lambda v: Mm @ v, m=kmax, tol=1e-14, max_iter=kmax)
    ref = _min_residuals(A, Mm, b, kmax)
    hist = np.array(info["history"][:kmax])
    assert np.allclose(hist, ref, rtol=1e-9, atol=1e-13)
    # the returned iterate attains the last minimum (true residual, recomputed)
    assert abs(np.linalg.norm(b - A @ x) / np.linalg.norm(b) - ref[-1]) <= 1e-9 * max(ref[-1], 1e-12)


def test_finite_termination_with_four_distinct_eigenvalues():
    rng = np.random.default_rng(9)
    X = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    lam = np.repeat(np.array([1.0 + 2.0j, -2.0 + 0.5j, 3.0, 0.5 - 1.0j]), N // 4)
    A = X @ np.diag(lam) @ np.linalg.inv(X)
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    x, info = G.gmres(lambda v: A @ v, b, lambda v: v, m=N, tol=1e-10, max_iter=N)
    assert info["converged"] and info["iters"] <= 4
    assert np.linalg.norm(A @ x - b) <= 1e-8 * np.linalg.norm(b)


def test_restarts_keep_the_true_residual_and_converge():
    A, Mm, b = _system(4)
    x, info = G.gmres(lambda v: A @ v, b, lambda v: Mm @ v, m=3, tol=1e-10, max_iter=200)
    assert info["converged"]
    assert abs(info["relres"] - np.linalg.norm(b - A @ x) / np.linalg.norm(b)) <= 1e-15
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-8 * np.linalg.norm(x)


# plausible mistakes planted in the oracle's own source: a Gram-Schmidt
# coefficient without the conjugate, a Givens rotation of the right-hand side
# without the conjugate, the previous rotations not applied to a new column
PLANTS = {
    "gram_schmidt_no_conjugate": ("np.vdot(V[i], w)", "np.dot(V[i], w)"),
    "rhs_rotation_no_conjugate": ("g[j + 1] = -np.conj(s) * g[j]", "g[j + 1] = -s * g[j]"),
    "previous_rotations_skipped": ("for i in range(j):                           # previous rotations",
                                   "for i in range(0):                           # previous rotations"),
}


def _planted_gmres(flaw):
    old, new = PLANTS[flaw]
    src = inspect.getsource(G.gmres)
    assert src.count(old) == 1, flaw
    ns = {"np": np, "givens": G.givens}
    exec(textwrap.dedent(src.replace(old, new)), ns)
    return ns["gmres"]


@pytest.mark.parametrize("flaw", sorted(PLANTS))
def test_planted_mistakes_fail_the_krylov_minimum(flaw):
    """Each plant breaks the reported history or the iterate's true residual
    (a rotation without the conjugate keeps the magnitudes of the history and
    spoils the iterate)."""
    A, Mm, b = _system(1)
    kmax = 6
    x, info = _planted_gmres(flaw)(lambda v: A @ v, b, lambda v: Mm @ v, m=kmax, tol=1e-14,
                                   max_iter=kmax)
    ref = _min_residuals(A, Mm, b, kmax)
    hist_ok = np.allclose(np.array(info["history"][:kmax]), ref, rtol=1e-6, atol=1e-10)
    true_res = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    iterate_ok = abs(true_res - ref[-1]) <= 1e-6 * max(ref[-1], 1e-12)
    assert not (hist_ok and iterate_ok)
