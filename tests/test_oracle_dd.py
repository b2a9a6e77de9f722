"""Pins of the oracle's domain decomposition, GMRES and two-grid cycle.

* J = 1: the sweeping preconditioner is an exact solve (T^(1) = tilde-T^(J) = 0,
  Section 2.1) -- any error in restriction/extension or the slab mesh shows;
* the preconditioners are linear maps (Section 2.1, text below Table 1);
* 1-D, constant k (Section 3.1): UD and X reproduce the solution up to the
  PML error, which shrinks as the DD PML widens;
* Theorem 1 (strip, constant k, PML in x, Dirichlet in y): A P_X f ~ f, so
  GMRES needs very few iterations;
* UD and X need about the same number of iterations (Table 7);
* GMRES returns A^-1 b to the tolerance; iteration counts stay roughly flat
  as omega grows at fixed points per wavelength (Section 6.1);
* the paper's printed iteration counts for TGSP and for the two-grid cycle
  with an exact coarse solve (Table 6, constant medium with PML).
"""

import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import dd, fd, gmres, mesh, twogrid
from oracle.problem import Problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dd_on(axes, k2, omega, J, w=4, s=20.0):
    A = fd.assemble(axes, k2, omega)
    builder = lambda ax, med: fd.assemble(ax, med, omega)   # noqa: E731
    return A, dd.SweepingDD(axes, k2, "node", builder, A, J, w, s, 1.0, omega)


def test_partition_eq17():
    beta, beta_t = dd.partition(101, 6)
    assert beta[0] == -1 and beta[-1] == 100 and beta_t[0] == -1 and beta_t[-1] == 100
    assert all(bt == b - 1 for b, bt in zip(beta[1:-1], beta_t[1:-1]))
    assert all(beta_t[j] < beta[j] < beta_t[j + 1] for j in range(1, 6))   # Eq. 8


def test_single_subdomain_is_exact_solve():
    cfg = synth.scaled_workload(2, 60, w_out=6, J=1)
    p = Problem(cfg, sweep="UD")
    rng = np.random.default_rng(4)
    f = rng.standard_normal(cfg.shape) + 1j * rng.standard_normal(cfg.shape)
    u = p.dd.apply(f, "UD")
    exact = spla.spsolve(p.A.tocsc(), f.ravel()).reshape(cfg.shape)
    assert np.abs(u - exact).max() <= 1e-10 * np.abs(exact).max()


@pytest.mark.parametrize("sweep", ["X", "UD"])
def test_preconditioner_is_linear(sweep):
    cfg = synth.scaled_workload(2, 60, w_out=6, J=4)
    p = Problem(cfg, sweep=sweep)
    rng = np.random.default_rng(5)
    f, g = (rng.standard_normal(cfg.shape) + 1j * rng.standard_normal(cfg.shape) for _ in range(2))
    a, b = 0.3 - 1.2j, 2.0 + 0.5j
    lhs = p.dd.apply(a * f + b * g, sweep)
    rhs = a * p.dd.apply(f, sweep) + b * p.dd.apply(g, sweep)
    assert np.abs(lhs - rhs).max() <= 1e-10 * np.abs(rhs).max()


@pytest.mark.parametrize("sweep", ["X", "UD"])
def test_one_dimensional_sweeps_are_nearly_exact(sweep):
    n, w_out = 600, 40
    h = 1.0 / n
    k = 2 * np.pi * 15.0
    ax = mesh.fine_axis(n + 2 * w_out, w_out, h, 20.0, 1.0)
    k2 = np.full(ax.N, k * k)
    rng = np.random.default_rng(6)
    f = rng.standard_normal(ax.N) + 1j * rng.standard_normal(ax.N)
    errs = []
    for w in (4, 8, 16):
        A, D = _dd_on([ax], k2, k, J=6, w=w, s=5.0 * w)
        u = D.apply(f, sweep)
        errs.append(np.linalg.norm(A @ u - f) / np.linalg.norm(f))
    assert errs[-1] < 1e-2
    assert errs[0] > errs[-1]


def test_theorem1_strip():
    nx, ny, w_out = 256, 31, 16
    h = 1.0 / nx
    k = 2 * np.pi * 10.0
    ax = mesh.fine_axis(nx + 2 * w_out, w_out, h, 20.0, 1.0)
    ay = mesh.fine_axis(ny + 1, 0, h, 20.0, 1.0)          # Dirichlet y-ends
    k2 = np.full((ay.N, ax.N), k * k)
    A, D = _dd_on([ay, ax], k2, k, J=6, w=8, s=40.0)
    rng = np.random.default_rng(7)
    f = rng.standard_normal(k2.shape) + 1j * rng.standard_normal(k2.shape)
    u = D.apply(f, "X")
    assert np.linalg.norm(A @ u.ravel() - f.ravel()) / np.linalg.norm(f) < 0.05
    x, info = gmres.gmres(lambda v: A @ v, f.ravel(), lambda v: D.apply(v, "X").ravel(), m=20)
    assert info["converged"] and info["iters"] <= 3


def test_gmres_matches_direct_solve_and_ud_x_agree():
    cfg = synth.scaled_workload(2, 200, w_out=12, J=8)
    b = synth.sources(cfg)[0]
    its = {}
    for sweep in ("X", "UD"):
        p = Problem(cfg, sweep=sweep)
        u, info = p.solve(b)
        exact = spla.spsolve(p.A.tocsc(), b.ravel())
        assert info["converged"] and info["relres"] <= cfg.tol
        assert np.linalg.norm(u.ravel() - exact) / np.linalg.norm(exact) < 1e-5
        assert np.linalg.norm(p.A @ u.ravel() - b.ravel()) / np.linalg.norm(b) <= 1.01 * cfg.tol
        its[sweep] = info["iters"]
    assert abs(its["X"] - its["UD"]) <= 2


def test_gmres_plain_against_dense_solve():
    rng = np.random.default_rng(8)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.3 + 1j * rng.standard_normal((n, n)) * 0.3
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, info = gmres.gmres(lambda v: A @ v, b, lambda v: v, m=10, tol=1e-10)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) / np.linalg.norm(x) < 1e-9
    c, s, r = gmres.givens(1 - 2j, 0.5 + 3j)
    v = np.array([c * (1 - 2j) + s * (0.5 + 3j), -np.conj(s) * (1 - 2j) + c * (0.5 + 3j)])
    assert abs(v[1]) < 1e-14 and abs(v[0] - r) < 1e-14 and abs(abs(r) - np.hypot(abs(1 - 2j), abs(0.5 + 3j))) < 1e-14


@pytest.mark.slow
def test_iterations_flat_in_frequency_at_fixed_ppw():
    its = []
    for n in (100, 200, 400):
        cfg = synth.scaled_workload(1, n, w_out=10, J=4)
        p = Problem(cfg)
        _, info = p.solve(synth.sources(cfg)[0])
        assert info["converged"]
        its.append(info["iters"])
    assert max(its) - min(its) <= 2


def _table6_workload(n, w, s):
    cells = n // 2 + 2 * 4
    J = cells // (2 * w + 1)
    J -= J % 2
    return synth.Workload(name="table6", dim=2, n=n, w_out=4, ppw=10.0, c_min=1.0,
                          medium="const", corr=0.0, J=J, w_dd=w, s_dd=s, s_out=20.0,
                          sweep="UD", two_grid=True, nu=3, omega_jac=0.8, gmres_m=30,
                          tol=1e-6, n_src=1, precision="fp64", seed=1)


@pytest.mark.slow
def test_table6_iteration_counts():
    rows = np.loadtxt(os.path.join(GOLDEN, "table6_constant_pml.txt"), dtype=int)
    for size, exact_its, *w_its in rows:
        if size > 256:
            continue
        for (w, s), paper in zip(((3, 15.0), (4, 20.0), (5, 25.0)), w_its):
            cfg = _table6_workload(int(size), w, s)
            p = Problem(cfg)
            b = synth.sources(cfg)[0]
            _, info = p.solve(b)
            assert abs(info["iters"] - paper) <= 2, (size, w, info["iters"], paper)
        lu = spla.splu(p.Ac.tocsc())
        M = lambda r: twogrid.tgsp(r.ravel(), p.A, p.P, lambda rc: lu.solve(rc), 3, 0.8).ravel()  # noqa: E731
        _, ie = gmres.gmres(p.apply, b.ravel(), M, m=30, tol=1e-6)
        assert abs(ie["iters"] - exact_its) <= 2


@pytest.mark.parametrize("flaw", ["transmission_sign", "tilde_transmission_dropped"])
def test_planted_mistakes_break_theorem1_pin(flaw, monkeypatch):
    """A wrong sign in Eq. 19 or a dropped Eq. 20 term must fail the strip pin."""
    if flaw == "transmission_sign":
        orig = dd.SweepingDD._T
        monkeypatch.setattr(dd.SweepingDD, "_T",
                            lambda self, j, B: tuple(-t for t in orig(self, j, B)))
    else:
        monkeypatch.setattr(dd.SweepingDD, "_Tt",
                            lambda self, j, B: (0 * B[1], 0 * B[0]))
    nx, ny, w_out = 256, 31, 16
    h = 1.0 / nx
    k = 2 * np.pi * 10.0
    ax = mesh.fine_axis(nx + 2 * w_out, w_out, h, 20.0, 1.0)
    ay = mesh.fine_axis(ny + 1, 0, h, 20.0, 1.0)
    k2 = np.full((ay.N, ax.N), k * k)
    A, D = _dd_on([ay, ax], k2, k, J=6, w=8, s=40.0)
    rng = np.random.default_rng(7)
    f = rng.standard_normal(k2.shape) + 1j * rng.standard_normal(k2.shape)
    u = D.apply(f, "X")
    assert np.linalg.norm(A @ u.ravel() - f.ravel()) / np.linalg.norm(f) > 0.2
