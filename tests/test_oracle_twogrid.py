"""Pins of the oracle's two-grid cycle (TGSP, Section 4; oracle/twogrid.py).

One cycle with zero initial guess is a linear map r -> M r.  Its error
propagation operator is fixed by the cycle's steps alone (Section 4.1:
nu omega-Jacobi pre-smoothing steps, residual restriction by R = P^T
(Section 4.2), a coarse correction with the coarse preconditioner C,
prolongation by P, nu post-smoothing steps):

    I - M A = (I - W A)^nu (I - P C P^T A) (I - W A)^nu,   W = omega_J D^-1.

The tests check the oracle against that identity on small dense complex
symmetric matrices, and against two consequences: with the Galerkin coarse
inverse C = (P^T A P)^-1 and no smoothing, the cycle solves exactly on the
coarse space (M A P = P), and with nu steps and no coarse correction it is
the textbook Jacobi polynomial.  A plausible mistake in the cycle (a
dropped post-smoothing, R = P^H in place of P^T for complex P, a wrong sign
of the correction) fails one of them.
"""

from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import twogrid

N, NC = 24, 7


def _case(seed):
    rng = np.random.default_rng(seed)
    # complex symmetric (A = A^T, not Hermitian) and diagonally dominant, like
    # the damped Helmholtz operators the cycle is applied to
    X = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    A = 0.1 * (X + X.T) + np.diag(6.0 + 1.0j + rng.random(N))
    P = rng.standard_normal((N, NC)) + 0.5j * rng.standard_normal((N, NC))
    return sp.csr_matrix(A), A, P


def _cycle_matrix(Asp, P, C, nu, omega):
    """Columns of M: the oracle's cycle applied to the unit vectors."""
    return np.stack([twogrid.tgsp(np.eye(N)[:, k].astype(complex), Asp, P, lambda rc: C @ rc,
                                  nu, omega) for k in range(N)], axis=1)


@pytest.mark.parametrize("nu", [0, 1, 3])
@pytest.mark.parametrize("galerkin", [True, False])
def test_error_propagation_identity(nu, galerkin):
    Asp, A, P = _case(1 + nu)
    omega = 0.8
    rng = np.random.default_rng(7)
    C = (np.linalg.inv(P.T @ A @ P) if galerkin else
         rng.standard_normal((NC, NC)) + 1j * rng.standard_normal((NC, NC)))
    M = _cycle_matrix(Asp, P, C, nu, omega)
    I = np.eye(N)
    S = np.linalg.matrix_power(I - omega * np.diag(1.0 / np.diag(A)) @ A, nu)
    E = S @ (I - P @ C @ P.T @ A) @ S
    assert np.abs((I - M @ A) - E).max() <= 1e-12 * max(1.0, np.abs(E).max())


def test_galerkin_coarse_space_is_solved_exactly_without_smoothing():
    Asp, A, P = _case(11)
    C = np.linalg.inv(P.T @ A @ P)
    M = _cycle_matrix(Asp, P, C, 0, 0.8)
    assert np.abs(M @ A @ P - P).max() <= 1e-12 * np.abs(P).max()


def test_smoothing_alone_is_the_jacobi_polynomial():
    """No coarse correction (C = 0): M = sum_{m < 2 nu} (I - W A)^m W."""
    Asp, A, P = _case(5)
    nu, omega = 2, 0.7
    M = _cycle_matrix(Asp, P, np.zeros((NC, NC)), nu, omega)
    W = omega * np.diag(1.0 / np.diag(A))
    G = np.eye(N) - W @ A
    ref = sum(np.linalg.matrix_power(G, m) @ W for m in range(2 * nu))
    assert np.abs(M - ref).max() <= 1e-12 * np.abs(ref).max()


def _flawed_tgsp(flaw):
    def cycle(r, A, P, coarse_prec, nu, omega_jac):
        r = r.ravel()
        dinv = 1.0 / A.diagonal()
        u = twogrid.jacobi(A, dinv, r, np.zeros_like(r, dtype=np.complex128), nu, omega_jac)
        R = P.conj().T if flaw == "hermitian_restriction" else P.T
        ec = coarse_prec(R @ (r - A @ u))
        u = u - P @ ec if flaw == "correction_sign" else u + P @ ec
        if flaw != "no_post_smoothing":
            u = twogrid.jacobi(A, dinv, r, u, nu, omega_jac)
        return u
    return cycle


@pytest.mark.parametrize("flaw", ["hermitian_restriction", "correction_sign", "no_post_smoothing"])
def test_planted_cycle_mistakes_fail_the_identity(flaw, monkeypatch):
    monkeypatch.setattr(twogrid, "tgsp", _flawed_tgsp(flaw))
    Asp, A, P = _case(3)
    nu, omega = 1, 0.8
    C = np.linalg.inv(P.T @ A @ P)
    M = _cycle_matrix(Asp, P, C, nu, omega)
    I = np.eye(N)
    S = np.linalg.matrix_power(I - omega * np.diag(1.0 / np.diag(A)) @ A, nu)
    E = S @ (I - P @ C @ P.T @ A) @ S
    assert np.abs((I - M @ A) - E).max() > 1e-6
