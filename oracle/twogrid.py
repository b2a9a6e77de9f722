"""Two-grid sweeping preconditioner, TGSP (Section 4).

One two-grid cycle with zero initial guess (Section 4.1): ``nu``
omega-Jacobi pre-smoothing steps u += omega_J D^-1 (r - A u) with
D = diag(A) (complex), restriction of the residual r_c = R (r - A u) with
R = P^T (Section 4.2), one sweeping-preconditioner application on the
coarse operator in place of the exact coarse solve (Section 4, first
paragraph), prolongation and correction u += P e_c, and ``nu``
post-smoothing steps.  The result is a linear map of r.
"""

from __future__ import annotations

import numpy as np


def jacobi(A, dinv, r, u, nu, omega_jac):
    for _ in range(nu):
        u = u + omega_jac * dinv * (r - A @ u)
    return u


def tgsp(r: np.ndarray, A, P, coarse_prec, nu: int, omega_jac: float) -> np.ndarray:
    shape = r.shape
    r = r.ravel()
    dinv = 1.0 / A.diagonal()
    u = np.zeros_like(r, dtype=np.complex128)
    u = jacobi(A, dinv, r, u, nu, omega_jac)
    rc = P.T @ (r - A @ u)
    ec = coarse_prec(rc)
    u = u + P @ ec.ravel()
    u = jacobi(A, dinv, r, u, nu, omega_jac)
    return u.reshape(shape)
