"""1-D meshes along one axis and the PML factors.

An axis with ``N`` unknowns has ``N + 1`` cells; cell ``c`` lies between
unknowns ``c - 1`` and ``c`` (cell 0 and cell N touch the Dirichlet nodes),
so the half point ``i - 1/2`` of the paper is cell ``i`` and ``i + 1/2`` is
cell ``i + 1``.  Each axis stores the cell sizes, the damping ``sigma`` at
the unknowns and at the cell midpoints.

PML (Section 2.1, Eqs. 4-5): d/dx -> (1 + i sigma/omega)^(-1) d/dx with
sigma = C_pml * d^2, d the distance into the layer, C_pml = S_pml * c_pml /
d_pml^3.  The factor used by the discretisations is
alpha = 1 / (1 + i sigma / omega) (definition below Eq. 40).
"""

from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Axis:
    h_cell: np.ndarray       # (N+1,) cell sizes
    sigma_node: np.ndarray   # (N,)   damping at the unknowns
    sigma_cell: np.ndarray   # (N+1,) damping at cell midpoints

    @property
    def N(self) -> int:
        return self.sigma_node.size

    def alpha_node(self, omega: float) -> np.ndarray:
        return 1.0 / (1.0 + 1j * self.sigma_node / omega)

    def alpha_cell(self, omega: float) -> np.ndarray:
        return 1.0 / (1.0 + 1j * self.sigma_cell / omega)


def pml_constant(s_pml: float, c_pml: float, d_pml: float) -> float:
    """C_pml = S_pml c_pml / d_pml^3 (text below Eq. 5)."""
    return s_pml * c_pml / d_pml ** 3


def fine_axis(n_cells: int, w_out: int, h: float, s_pml: float, c_pml: float) -> Axis:
    """Uniform axis of ``n_cells`` cells with ``w_out`` PML cells on both sides.

    Node p sits at x = p h; the interior box is [w_out h, (n_cells - w_out) h]
    and sigma grows quadratically with the distance beyond it (Eq. 5), with
    d_pml = w_out h.
    """
    C = pml_constant(s_pml, c_pml, w_out * h) if w_out > 0 else 0.0
    lo, hi = w_out * h, (n_cells - w_out) * h

    def sigma(x):
        d = np.maximum(0.0, np.maximum(lo - x, x - hi))
        return C * d * d

    x_node = np.arange(1, n_cells) * h
    x_mid = (np.arange(n_cells) + 0.5) * h
    return Axis(h_cell=np.full(n_cells, h), sigma_node=sigma(x_node), sigma_cell=sigma(x_mid))


def sponge_beta_max(damping: float, k_ref: float, width: float) -> float:
    """beta_max of a quadratic sponge profile beta(d) = beta_max (d / width)^2
    whose one-way amplitude damping exp(-int k beta dx) = exp(-k beta_max
    width / 3) equals `damping` at the wavenumber k_ref (Section 2.1: k is
    replaced by k (1 + i beta) in the sponge; reading: the damping is set at
    the typical wavenumber omega / c_pml)."""
    return 3.0 * np.log(1.0 / damping) / (k_ref * width)


def sponge_beta(n_cells: int, w_out: int, h: float, beta_max: float) -> np.ndarray:
    """beta at the unknowns of a uniform axis whose outer w_out cells on both
    sides form the sponge: quadratic in the distance beyond the interior box
    (the same geometry as the PML profile of Eq. 5), zero inside."""
    if w_out == 0:
        return np.zeros(n_cells - 1)
    lo, hi = w_out * h, (n_cells - w_out) * h
    x = np.arange(1, n_cells) * h
    d = np.maximum(0.0, np.maximum(lo - x, x - hi))
    return beta_max * (d / (w_out * h)) ** 2


def sponge_factor(betas: list) -> np.ndarray:
    """(1 + i beta)^2 on the tensor grid, beta = sum of the per-axis profiles
    (reading of beta(x, y)): k^2 -> k^2 (1 + i beta)^2."""
    import functools
    b = functools.reduce(np.add.outer, betas) if len(betas) > 1 else betas[0]
    return (1.0 + 1j * b) ** 2


def coarse_axis(n_int: int, w_out: int, h: float, s_pml: float, c_pml: float):
    """PML-aware coarsening of a fine axis (Section 4.2).

    The fine axis has ``w_out`` PML cells of size h on each side and ``n_int``
    interior cells.  PML cells are kept; interior cells are merged in pairs
    (size 2h).  Returns ``(axis, i_fp, refined)`` where ``i_fp[Q]`` maps a
    coarse node number Q (0..coarse cells) to the fine node number and
    ``refined[Q]`` tells whether coarse cell Q + 1/2 is refined (the function
    r_C of Section 4.2).  sigma is evaluated at the coarse nodes and at the
    coarse cell midpoints with the fine axis' profile.
    """
    assert n_int % 2 == 0
    n_c = 2 * w_out + n_int // 2
    Q = np.arange(n_c + 1)
    i_fp = np.where(Q <= w_out, Q,
                    np.where(Q <= w_out + n_int // 2, w_out + 2 * (Q - w_out), Q + n_int // 2))
    refined = (Q >= w_out) & (Q < w_out + n_int // 2)
    x = i_fp * h
    C = pml_constant(s_pml, c_pml, w_out * h) if w_out > 0 else 0.0
    lo, hi = w_out * h, (2 * w_out + n_int - w_out) * h

    def sigma(xx):
        d = np.maximum(0.0, np.maximum(lo - xx, xx - hi))
        return C * d * d

    h_cell = np.diff(x)
    x_mid = 0.5 * (x[:-1] + x[1:])
    axis = Axis(h_cell=h_cell.astype(np.float64), sigma_node=sigma(x[1:-1]), sigma_cell=sigma(x_mid))
    return axis, i_fp, refined[:-1]
