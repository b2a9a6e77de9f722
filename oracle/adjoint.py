"""Adjoint gradient of a receiver misfit (not in the paper; defined from Eq. 40).

Misfit: Phi(m) = 1/2 sum_s sum_q |u_s(x_q) - d_{s,q}|^2 with A(m) u_s = b_s,
A the h^d-scaled Eq. 40 and b_s independent of m.  Only the mass term of Eq. 40
depends on m (k^2 = omega^2 m s, s = (1 + i beta)^2 in a sponge layer of
Section 2.1, else 1): dA/dm_i = -omega^2 w_i e_i e_i^T with
w_i = h^d s_i / prod_l alpha_{l,i}.  The PML and sponge parameters (c_pml) are
held fixed.
With r_s = R u_s - d_s (R: sampling at the receivers) and A complex symmetric,
mu_s solving A mu_s = conj(R^T r_s) gives

    dPhi/dm_i = omega^2 Re( w_i sum_s mu_{s,i} u_{s,i} ).

The solves here are exact sparse LU solves (library primitive).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import fd


def misfit_and_gradient(problem, src_nodes_flat, rec_flat, d_obs):
    """(Phi, grad) for point sources b_s = e_{src_s} (flat indices) and receivers rec_flat."""
    A = problem.A.tocsc()
    lu = spla.splu(A)
    n = A.shape[0]
    # h^d s / prod alpha
    w = (fd.rhs_scaling(problem.axes, problem.omega) * problem.sponge).ravel()
    phi = 0.0
    grad = np.zeros(n)
    us = []
    for s, node in enumerate(src_nodes_flat):
        b = np.zeros(n, complex)
        b[node] = 1.0
        u = lu.solve(b)
        us.append(u)
        r = u[rec_flat] - d_obs[s]
        phi += 0.5 * float(np.sum(np.abs(r) ** 2))
        a = np.zeros(n, complex)
        np.add.at(a, rec_flat, np.conj(r))
        mu = lu.solve(a)
        grad += problem.omega ** 2 * np.real(w * mu * u)
    return phi, grad.reshape(problem.cfg.shape), us


def synthetic_data(problem_true, src_nodes_flat, rec_flat):
    """Receiver data of the true model (exact solves)."""
    lu = spla.splu(problem_true.A.tocsc())
    n = problem_true.A.shape[0]
    out = []
    for node in src_nodes_flat:
        b = np.zeros(n, complex)
        b[node] = 1.0
        out.append(lu.solve(b)[rec_flat])
    return np.array(out)
