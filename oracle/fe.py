"""Coarse-level optimised finite-element operator with PML (Appendix A).

* Table 9: the coefficients c_j(1/G_k) of the optimised finite differences,
  linearly interpolated in 1/G (Appendix A.1), G = 2 pi / (h k).
* Eq. 63: the mass / stiffness constants I_a, J_b chosen so that interior
  rows equal h^d times H_FDOpt (Eq. 47).  3-D as printed; 2-D is the
  analogue for the three-coefficient 2-D family (reading: mass weights
  c1 N0 + c2 N1 + (1-c1-c2) N2 and transverse averaging c3 + (1-c3) A1), i.e.
  I0 = c1/4, I1 = c2/8, I2 = (1-c1-c2)/4, J0 = c3/2, J1 = (1-c3)/2.
* Eqs. 53-61: H_FE = -M_FE - sum_l D^(l) (x) N^(others), written here as the
  equivalent sum over cells (cellwise-constant k^2, alpha and c_j): a cell
  with corners a, b contributes
      -vol * I_{|a-b|} * k^2 / prod(alpha)                        (mass, Eq. 54)
      - sum_l sgn_l * (alpha_l / h_l) * prod_{m!=l} (h_m / alpha_m)
              * J_{|a-b| over axes m != l}                         (Eqs. 59-61)
  with sgn_l = -1 if a_l == b_l else +1 (the per-cell part of D_{2,FE}).
* Section 4.2 / Eqs. 41-42: prolongation by tent functions on the
  PML-aware coarse mesh; restriction R = P^T.
* Appendix A.3, last paragraph: coarse-cell k^2 by tensor averaging of the
  fine nodal values, weights (1/2, 1/2) across unrefined cells and
  (1/4, 1/2, 1/4) across refined ones (reading: k^2 is averaged).
"""

from __future__ import annotations

import functools
import itertools

import numpy as np
import scipy.sparse as sp

from .mesh import Axis

# Table 9 (a): 2-D, columns 1/G_k, c1, c2, c3
TABLE9_2D = np.array([
    [0.00, 0.61953, 0.45295, 0.77363],
    [0.04, 0.63691, 0.47535, 0.87242],
    [0.08, 0.62988, 0.48633, 0.86400],
    [0.12, 0.62610, 0.48880, 0.84984],
    [0.16, 0.62289, 0.48759, 0.83017],
    [0.20, 0.62596, 0.47106, 0.80852],
    [0.24, 0.62213, 0.46478, 0.78215],
    [0.28, 0.61036, 0.47016, 0.74857],
    [0.32, 0.59107, 0.48468, 0.70553],
    [0.36, 0.56369, 0.50746, 0.65062],
    [0.40, 0.52412, 0.54163, 0.57676],
])

# Table 9 (b): 3-D, columns 1/G_k, c1 .. c5
TABLE9_3D = np.array([
    [0.00, 0.56428, 0.35970, 0.20490, 0.77998, 0.17505],
    [0.04, 0.56571, 0.36071, 0.20541, 0.78635, 0.17442],
    [0.08, 0.56298, 0.36150, 0.20719, 0.78273, 0.16881],
    [0.12, 0.56540, 0.35620, 0.20287, 0.76438, 0.18678],
    [0.16, 0.56370, 0.35299, 0.20299, 0.74684, 0.19603],
    [0.20, 0.55813, 0.35277, 0.20452, 0.72755, 0.20131],
    [0.24, 0.54673, 0.35830, 0.20693, 0.70298, 0.20847],
    [0.28, 0.52423, 0.38368, 0.19633, 0.66863, 0.22424],
    [0.32, 0.49946, 0.39740, 0.20725, 0.62734, 0.23845],
    [0.36, 0.47567, 0.40216, 0.22132, 0.58198, 0.25329],
    [0.40, 0.45011, 0.36784, 0.29962, 0.53417, 0.23589],
])


def coefficients(inv_G, dim: int):
    """c_j(1/G) by linear interpolation in Table 9; 1/G clamped to [0, 0.40]."""
    tab = TABLE9_2D if dim == 2 else TABLE9_3D
    x = np.clip(inv_G, 0.0, 0.40)
    return [np.interp(x, tab[:, 0], tab[:, j]) for j in range(1, tab.shape[1])]


def fe_constants(c, dim: int):
    """(I_0..I_d, J_0..J_{d-1}) from c_j: Eq. 63 (3-D) and its 2-D analogue."""
    if dim == 3:
        c1, c2, c3, c4, c5 = c
        I = [c1 / 8, c2 / 24, c3 / 24, (1 - c1 - c2 - c3) / 8]
        J = [c4 / 4, c5 / 8, (1 - c4 - c5) / 4]
    elif dim == 2:
        c1, c2, c3 = c
        I = [c1 / 4, c2 / 8, (1 - c1 - c2) / 4]
        J = [c3 / 2, (1 - c3) / 2]
    else:
        raise ValueError("the optimised coarse operator is defined for 2-D and 3-D")
    return I, J


def _bc(v, l, d):
    shape = [1] * d
    shape[l] = v.size
    return v.reshape(shape)


def _stiff_factor(alpha_cell: np.ndarray, h_cell: np.ndarray) -> np.ndarray:
    """alpha_l / h_l: the factor of the differentiated axis in the cell sum (Eqs. 59-61)."""
    return alpha_cell / h_cell


def _other_factor(alpha_cell: np.ndarray, h_cell: np.ndarray) -> np.ndarray:
    """h_m / alpha_m: the factor of every other axis in the cell sum (Eqs. 59-61)."""
    return h_cell / alpha_cell


def assemble(axes: list[Axis], k2cell: np.ndarray, omega: float, H: float,
             coeffs=None) -> sp.csr_matrix:
    """H_FE (Eq. 61) on the rectilinear mesh ``axes`` with cellwise k^2.

    ``k2cell`` has shape (N_0+1, ..., N_{d-1}+1); ``H`` is the reference
    spacing used in G = 2 pi / (H k) for the per-cell coefficients.
    ``coeffs`` (tests only) replaces the Table 9 values c_j by fixed ones;
    c = (4/9, 4/9, 2/3) in 2-D and (8/27, 4/9, 2/9, 4/9, 4/9) in 3-D give the
    constants of exactly integrated multilinear elements.
    """
    d = len(axes)
    Ns = [ax.N for ax in axes]
    cshape = tuple(n + 1 for n in Ns)
    assert k2cell.shape == cshape
    hc = [ax.h_cell for ax in axes]
    ac = [ax.alpha_cell(omega) for ax in axes]
    vol = functools.reduce(np.multiply, [_bc(hc[l], l, d) for l in range(d)])
    palpha = functools.reduce(np.multiply, [_bc(ac[l], l, d) for l in range(d)])
    # G from the cell's wavenumber; in a sponge (complex k^2 = k^2 (1 + i beta)^2)
    # from its real part k (reading: the damping does not change the coefficients)
    inv_G = H * np.real(np.sqrt(k2cell.astype(np.complex128))) / (2.0 * np.pi)
    c = coefficients(inv_G, d) if coeffs is None else [np.full(cshape, float(v)) for v in coeffs]
    I, Jc = fe_constants(c, d)
    mass = vol * k2cell / palpha
    idx = np.indices(cshape)
    rows, cols, vals = [], [], []
    for a in itertools.product((0, 1), repeat=d):
        for b in itertools.product((0, 1), repeat=d):
            ham = sum(int(a[l] != b[l]) for l in range(d))
            val = -I[ham] * mass
            for l in range(d):
                ham_o = sum(int(a[m] != b[m]) for m in range(d) if m != l)
                sgn = -1.0 if a[l] == b[l] else 1.0
                other = functools.reduce(np.multiply, [_bc(_other_factor(ac[m], hc[m]), m, d)
                                                       for m in range(d) if m != l], 1.0)
                val = val - sgn * _bc(_stiff_factor(ac[l], hc[l]), l, d) * other * Jc[ham_o]
            val = np.broadcast_to(val, cshape)
            ia = [idx[l] + a[l] - 1 for l in range(d)]
            ib = [idx[l] + b[l] - 1 for l in range(d)]
            ok = np.ones(cshape, dtype=bool)
            for l in range(d):
                ok &= (ia[l] >= 0) & (ia[l] < Ns[l]) & (ib[l] >= 0) & (ib[l] < Ns[l])
            rows.append(np.ravel_multi_index([x[ok] for x in ia], Ns))
            cols.append(np.ravel_multi_index([x[ok] for x in ib], Ns))
            vals.append(val[ok])
    n = int(np.prod(Ns))
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n)).tocsr()


def averaging_1d(i_fp: np.ndarray, refined: np.ndarray, n_fine_cells: int) -> np.ndarray:
    """Rows: coarse cells; columns: fine nodes 0..n_fine_cells (Appendix A.3)."""
    n_c = refined.size
    W = np.zeros((n_c, n_fine_cells + 1))
    for Q in range(n_c):
        p = i_fp[Q]
        if refined[Q]:
            W[Q, p:p + 3] = (0.25, 0.5, 0.25)
        else:
            W[Q, p:p + 2] = (0.5, 0.5)
    return W


def coarse_k2(k2_fine: np.ndarray, i_fp, refined) -> np.ndarray:
    """Coarse cellwise k^2 from fine nodal k^2 (edge values copied to the Dirichlet nodes).

    ``i_fp`` / ``refined`` describe one axis (used for all) or are lists with
    one entry per array axis.
    """
    d = k2_fine.ndim
    if not isinstance(i_fp, (list, tuple)):
        i_fp, refined = [i_fp] * d, [refined] * d
    kp = np.pad(k2_fine, 1, mode="edge")
    out = kp
    for l in range(d):
        W = averaging_1d(i_fp[l], refined[l], kp.shape[l] - 1)
        out = np.moveaxis(np.tensordot(W, np.moveaxis(out, l, 0), axes=(1, 0)), 0, l)
    return out


def prolongation_1d(i_fp: np.ndarray, refined: np.ndarray, n_fine: int) -> sp.csr_matrix:
    """Eqs. 41-42: (P u)_{i_FP(Q)} = u_Q; (P u)_{i_FP(Q)+1} = (u_Q + u_{Q+1})/2 if r_C(Q+1/2).

    Coarse unknown q is coarse node Q = q + 1; fine unknown = fine node - 1;
    Dirichlet nodes carry zero.
    """
    n_c = refined.size
    rows, cols, vals = [], [], []
    for Q in range(1, n_c):
        rows.append(i_fp[Q] - 1); cols.append(Q - 1); vals.append(1.0)
    for Q in range(n_c):
        if refined[Q]:
            p = i_fp[Q] + 1
            if Q >= 1:
                rows.append(p - 1); cols.append(Q - 1); vals.append(0.5)
            if Q + 1 <= n_c - 1:
                rows.append(p - 1); cols.append(Q); vals.append(0.5)
    return sp.coo_matrix((vals, (rows, cols)), shape=(n_fine, n_c - 1)).tocsr()


def prolongation(p1d: list) -> sp.csr_matrix:
    """Tensor product of the 1-D prolongations (Section 4.2)."""
    return functools.reduce(lambda a, b: sp.kron(a, b, format="csr"), p1d)
