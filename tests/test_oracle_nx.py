"""Pins of the oracle's NX-sweep (SweepingPrecNX, Table 3; partial sweeps).

* With one cell the NX-sweep is the X-sweep, exactly (j_cell = 0, J + 1).
* It is a linear map.
* In 1-D with constant k the PML transmission is nearly exact, and one
  NX application carries waves across at most one cell boundary: for f
  inside a cell the output is nearly exact on that cell and its boundary
  subdomains, for f in a cell
  boundary subdomain on both neighbouring cells (the error shrinks as the DD
  PML widens), while it is not a global inverse.  A wrong wiring of the
  cell boundaries (the final boundary solve without the left cell's layers)
  breaks the pin.
* Table 7 of the paper (constant medium): the partial sweeps need more GMRES
  iterations than the X-sweep, and more as the cell count grows.
"""

import numpy as np
import pytest

import scipy.sparse.linalg as spla

import synth
from oracle import dd, fd, mesh
from oracle.problem import Problem


def _dd_on(axes, k2, omega, J, w=4, s=20.0):
    A = fd.assemble(axes, k2, omega)
    builder = lambda ax, med: fd.assemble(ax, med, omega)   # noqa: E731
    return A, dd.SweepingDD(axes, k2, "node", builder, A, J, w, s, 1.0, omega)


def test_layout():
    assert dd.nx_layout(16, 1) == ([0, 17], [0, 9])       # the X-sweep's j_mid = J/2 + 1
    jc, jm = dd.nx_layout(16, 4)
    assert jc[0] == 0 and jc[-1] == 17 and len(jc) == 5
    assert all(jc[m - 1] < jm[m] < jc[m] for m in range(1, 5))
    with pytest.raises(AssertionError):
        dd.nx_layout(4, 3)


def test_one_cell_is_the_x_sweep():
    cfg = synth.scaled_workload(2, 60, w_out=6, J=6)
    p = Problem(cfg)
    f = np.random.default_rng(1).standard_normal(cfg.shape) + 0.5j
    assert np.array_equal(p.dd.prec_nx(f, 1), p.dd.prec_x(f))


def test_nx_is_linear():
    cfg = synth.scaled_workload(2, 60, w_out=6, J=6)
    p = Problem(cfg)
    rng = np.random.default_rng(5)
    f, g = (rng.standard_normal(cfg.shape) + 1j * rng.standard_normal(cfg.shape) for _ in range(2))
    a, b = 0.3 - 1.2j, 2.0 + 0.5j
    lhs = p.dd.prec_nx(a * f + b * g, 2)
    rhs = a * p.dd.prec_nx(f, 2) + b * p.dd.prec_nx(g, 2)
    assert np.abs(lhs - rhs).max() <= 1e-10 * np.abs(rhs).max()


def _cols(D, j0, j1):
    """Global columns owned by subdomains j0..j1 (forward intervals, Eq. 17)."""
    return np.arange(D.beta[j0 - 1] + 1, D.beta[j1] + 1)


def _errs_1d(where, n_cell=3, ws=(4, 8, 16)):
    """Relative error of the NX output against the exact solution, on the cells
    that f's support can reach in one application: f inside cell 2 (error on
    cell 2 and its two boundary subdomains), or f in the cell boundary
    subdomain j_cell[1] (error on cells 1 and 2 and the boundary subdomain)."""
    n, w_out = 600, 40
    h = 1.0 / n
    k = 2 * np.pi * 15.0
    ax = mesh.fine_axis(n + 2 * w_out, w_out, h, 20.0, 1.0)
    k2 = np.full(ax.N, k * k)
    J = 9
    jc, jm = dd.nx_layout(J, n_cell)
    rng = np.random.default_rng(6)
    errs = []
    for w in ws:
        A, D = _dd_on([ax], k2, k, J=J, w=w, s=5.0 * w)
        f = np.zeros(ax.N, complex)
        if where == "cell":
            # cell 2, its left boundary subdomain and the columns of its right
            # boundary subdomain that the second-phase MidSolveIn writes
            # (the last one belongs to the next cell's backward sweep)
            src = _cols(D, jc[1] + 1, jc[2] - 1)
            seen = np.concatenate([_cols(D, jc[1], jc[2] - 1),
                                   np.arange(D.beta[jc[2] - 1] + 1, D.beta_t[jc[2]] + 1)])
        else:
            src, seen = _cols(D, jc[1], jc[1]), _cols(D, jc[0] + 1, jc[2] - 1)
        f[src] = rng.standard_normal(src.size) + 1j * rng.standard_normal(src.size)
        u = D.prec_nx(f, n_cell)
        exact = spla.spsolve(A.tocsc(), f)
        errs.append(np.linalg.norm((u - exact)[seen]) / np.linalg.norm(exact[seen]))
    return errs


@pytest.mark.parametrize("where", ["cell", "boundary"])
def test_one_dimensional_nx_is_exact_on_the_reached_cells(where):
    errs = _errs_1d(where)
    assert errs[-1] < 1e-2
    assert errs[0] > errs[-1]


def test_one_dimensional_nx_is_not_a_global_inverse():
    """Waves do not cross a second cell boundary in one application."""
    n, w_out, k = 600, 40, 2 * np.pi * 15.0
    ax = mesh.fine_axis(n + 2 * w_out, w_out, 1.0 / n, 20.0, 1.0)
    A, D = _dd_on([ax], np.full(ax.N, k * k), k, J=9, w=16, s=80.0)
    f = np.random.default_rng(2).standard_normal(ax.N) + 0j
    u = D.prec_nx(f, 3)
    assert np.linalg.norm(A @ u - f) / np.linalg.norm(f) > 0.1


def test_planted_one_way_boundary_fails(monkeypatch):
    """A second-phase MidSolveIn of a cell boundary wired to the right cell's
    data only (the left cell's forward layers dropped) leaves the boundary
    subdomain without the left cell's waves.  (A first-phase boundary
    MidSolveOut sending one way only is repaired by the residual phase, so
    it is not a discriminating mistake.)"""
    real = dd.SweepingDD.mid_solve_in
    jc, _ = dd.nx_layout(9, 3)

    def right_only(self, u, f, j, B1, B2):   # cell boundaries: second phase only
        if j in jc[1:-1]:
            B1 = [np.zeros_like(B1[0]), np.zeros_like(B1[1])]
        real(self, u, f, j, B1, B2)

    monkeypatch.setattr(dd.SweepingDD, "mid_solve_in", right_only)
    assert _errs_1d("cell", ws=(16,))[-1] > 1e-1


def test_table7_partial_sweeps_need_more_iterations():
    cfg = synth.scaled_workload(1, 120, w_out=8, J=12)
    b = synth.sources(cfg)[0]
    its = {}
    for sweep, nc in (("X", 1), ("NX", 2), ("NX", 4)):
        _, info = Problem(cfg, sweep=sweep, n_cell=nc).solve(b)
        assert info["converged"]
        its[(sweep, nc)] = info["iters"]
    assert its[("X", 1)] < its[("NX", 2)] <= its[("NX", 4)]
