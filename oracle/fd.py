"""Fine-grid finite-difference Helmholtz operator with PML (Eq. 40).

Eq. 40 (2-D) discretises -(1/a2) d_x(a1 d_x u) - (1/a1) d_y(a2 d_y u)
- k^2/(a1 a2) u with the 1-D three-point rule of Eq. 39, a_l the PML factor
of axis l.  Reading of the garbled mass term: it multiplies u_{i,k}.  The
same construction in d dimensions (3-point in 1-D, 7-point in 3-D) is

    (A u)_i = sum_l h^(d-2) prod_{m != l} (1/a_{m,i_m})
                    * (-a_{l,i-1/2} u_{i-e_l} + (a_{l,i-1/2} + a_{l,i+1/2}) u_i
                       - a_{l,i+1/2} u_{i+e_l})
              - h^d k_i^2 / prod_m a_{m,i_m} * u_i ,

i.e. Eq. 40 multiplied by h^d (the finite-element-like scaling of Appendix
A.3).  The right-hand side of this system is h^d f / prod_m a_m; a unit
point source (f = h^-d at an interior node) is b = 1 there.  The matrix is
complex symmetric.
"""

from __future__ import annotations

import functools

import numpy as np
import scipy.sparse as sp

from .mesh import Axis


def _kron_all(mats):
    return functools.reduce(lambda a, b: sp.kron(a, b, format="csr"), mats)


def second_difference(alpha_cell: np.ndarray) -> sp.csr_matrix:
    """1-D matrix of Eq. 39 with beta = alpha at the half points (without 1/h^2).

    Row i: -a_{i-1/2} u_{i-1} + (a_{i-1/2} + a_{i+1/2}) u_i - a_{i+1/2} u_{i+1};
    a_{i-1/2} is ``alpha_cell[i]`` and a_{i+1/2} is ``alpha_cell[i+1]``.
    """
    a = alpha_cell
    return sp.diags([-a[1:-1], a[:-1] + a[1:], -a[1:-1]], [-1, 0, 1], format="csr")


def assemble(axes: list[Axis], k2: np.ndarray, omega: float) -> sp.csr_matrix:
    """h^d-scaled Eq. 40 on the tensor mesh ``axes`` (array-axis order, x last).

    ``k2`` holds k^2 = omega^2 m at the unknowns, shape (N_0, ..., N_{d-1}).
    """
    d = len(axes)
    h = float(axes[0].h_cell[0])
    for ax in axes:
        assert np.allclose(ax.h_cell, h), "finite differences need a uniform mesh"
    an = [ax.alpha_node(omega) for ax in axes]
    ac = [ax.alpha_cell(omega) for ax in axes]
    A = None
    for l in range(d):
        mats = [second_difference(ac[m]) if m == l else sp.diags(1.0 / an[m]) for m in range(d)]
        term = h ** (d - 2) * _kron_all(mats)
        A = term if A is None else A + term
    prod_alpha = functools.reduce(np.multiply.outer, an) if d > 1 else an[0]
    mass = h ** d * k2.reshape(prod_alpha.shape) / prod_alpha
    return (A - sp.diags(mass.ravel())).tocsr()


def rhs_scaling(axes: list[Axis], omega: float) -> np.ndarray:
    """h^d / prod_m a_m at the unknowns: b = rhs_scaling * f (right side of Eq. 40)."""
    d = len(axes)
    h = float(axes[0].h_cell[0])
    an = [ax.alpha_node(omega) for ax in axes]
    prod_alpha = functools.reduce(np.multiply.outer, an) if d > 1 else an[0]
    return h ** d / prod_alpha
