"""Sponge boundary layers on the GPU against the oracle.

Section 2.1: in an outer sponge layer k is replaced by k (1 + i beta), beta
quadratic in the depth, and there is no PML (alpha = 1); Section 4.1: the
two-grid cycle then coarsens every cell (standard coarsening), so the coarse
cell k^2 is complex and the Table 9 coefficients are read at Re k.  Checked
here: the fine operator (2-D and 3-D), the slab solves (the added DD PML
freezes the complex k^2 of the interface cell), the fine-grid and two-grid
sweeping preconditioners (X and UD), GMRES against the oracle's direct solve,
the adjoint gradient (dA/dm carries the sponge factor) and the "Constant
medium, sponge" block of Table 6 (tests/golden/table6_constant_sponge.txt).

Tolerances as in the PML parity tests: FP64 operators 1e-12, FP64 slab
solves and preconditioners 1e-9, complex64 3e-4, GMRES solutions 1e-5.
"""

import dataclasses
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import adjoint
from oracle.problem import Problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-9, "mixed": 3e-4}
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hz():
    import paper_1412_0464_gb300 as hz
    hz.build()
    return hz


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def _close(a, b, tol):
    return _rel(a, b) <= tol and np.abs(a - b).max() <= tol * np.abs(b).max()


def _cfg(idx, n, w_out, J, **over):
    return synth.scaled_workload(idx, n, w_out=w_out, J=J, boundary="sponge", **over)


# (config, n, w_out, J, two_grid): 2-D fine-grid sweeps (config 2 recipe, ragged
# slabs), 2-D two-grid, 3-D fine-grid (config 4 recipe) and 3-D two-grid (config 5)
CASES = [(2, 64, 12, 6, False), (2, 72, 14, 4, True), (4, 14, 5, 2, False), (5, 20, 6, 2, True)]


@pytest.mark.parametrize("idx,n,w_out,J,two_grid", CASES)
def test_sponge_apply_matches_oracle(idx, n, w_out, J, two_grid):
    hz = _hz()
    cfg = _cfg(idx, n, w_out, J, n_src=2, two_grid=two_grid)
    p = Problem(cfg)
    s = hz.Solver.from_workload(cfg, precision="fp64")
    u = _rand((2,) + cfg.shape, 1)
    y = s.apply(torch.from_numpy(u).cuda()).cpu().numpy()
    for r in range(2):
        ref = (p.A @ u[r].ravel()).reshape(cfg.shape)
        assert np.abs(y[r] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("idx,n,w_out,J,two_grid", CASES)
def test_sponge_slab_solves_match_oracle(idx, n, w_out, J, two_grid, precision):
    hz = _hz()
    cfg = _cfg(idx, n, w_out, J, n_src=2, two_grid=two_grid)
    p = Problem(cfg)
    s = hz.Solver.from_workload(cfg, precision=precision)
    s.factor()
    for j in range(1, J + 1):
        sl = p.dd.slabs[j]
        info = s.slab_info(j)
        assert (info["lo"], info["hi"], info["wl"], info["wr"], info["W"]) == \
            (sl.lo, sl.hi, sl.wl, sl.wr, sl.W)
        nt = sl.A.shape[0] // sl.W
        assert nt == s.slab_nt
        fd = _rand((2, nt, sl.W), 10 + j)
        ud = s.slab_solve(j, torch.from_numpy(fd).cuda()).cpu().numpy()
        for r in range(2):
            ref = sl.lu.solve(fd[r].ravel()).reshape(nt, sl.W)
            assert _close(ud[r], ref, TOL[precision]), (j, r, _rel(ud[r], ref))


@pytest.mark.parametrize("sweep", ["X", "UD"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("idx,n,w_out,J,two_grid", CASES)
def test_sponge_preconditioner_matches_oracle(idx, n, w_out, J, two_grid, precision, sweep):
    if sweep == "X" and J % 2:
        pytest.skip("the X-sweep needs an even J")
    hz = _hz()
    cfg = _cfg(idx, n, w_out, J, n_src=2, two_grid=two_grid)
    p = Problem(cfg, sweep=sweep)
    s = hz.Solver.from_workload(cfg, precision=precision, sweep=sweep)
    s.factor()
    f = _rand((2,) + cfg.shape, 3)
    z = s.precond(torch.from_numpy(f).cuda()).cpu().numpy()
    for r in range(2):
        assert _close(z[r], p.precondition(f[r]).reshape(cfg.shape), TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("idx,n,w_out,J,two_grid", [CASES[1], CASES[3]])
def test_sponge_solve_matches_direct_solve(idx, n, w_out, J, two_grid, precision):
    hz = _hz()
    cfg = _cfg(idx, n, w_out, J, n_src=2, two_grid=two_grid)
    p = Problem(cfg)
    s = hz.Solver.from_workload(cfg, precision=precision, sweep="UD")
    s.factor()
    b = synth.sources(cfg)[:2]
    u, st = s.solve(torch.from_numpy(b).cuda())
    u = u.cpu().numpy()
    lu = spla.splu(p.A.tocsc())
    for r in range(2):
        assert _rel(u[r], lu.solve(b[r].ravel()).reshape(cfg.shape)) <= 1e-5
    assert st["relres_max"] <= cfg.tol


def test_sponge_gradient_matches_oracle():
    hz = _hz()
    cfg = dataclasses.replace(synth.adjoint_workload_2d(64), boundary="sponge", w_out=12)
    m_true, m0 = synth.medium(cfg, "true"), synth.medium(cfg, "start")
    c_pml = float(np.mean(1.0 / np.sqrt(m0)))
    src = np.array([int(i) * cfg.N + int(j) for i, j in synth.source_nodes(cfg)])
    rec = synth.receivers(cfg)
    d = adjoint.synthetic_data(Problem(cfg, m_true, two_grid=False, c_pml=c_pml), src, rec)
    s = hz.Solver.from_workload(cfg, m=m0, tol=1e-10, c_pml=c_pml, max_rhs=4)
    s.factor()
    phi, g, st = s.grad(src, rec, d)
    phi_o, g_o, _ = adjoint.misfit_and_gradient(Problem(cfg, m0, two_grid=False, c_pml=c_pml),
                                                src, rec, d)
    g = g.cpu().numpy()
    assert phi > 0 and abs(phi - phi_o) <= 1e-8 * phi_o
    assert np.abs(g - g_o).max() <= 1e-7 * np.abs(g_o).max()
    assert st["relres_max"] <= 1e-10


def _table6_sponge(n, w, s):
    cells = n // 2 + 36                        # coarse cells across, sponge included
    J = cells // (2 * w + 1)
    J -= J % 2
    return synth.Workload(name="table6s", dim=2, n=n, w_out=36, ppw=10.0, c_min=1.0,
                          medium="const", corr=0.0, J=J, w_dd=w, s_dd=s, s_out=20.0,
                          sweep="UD", two_grid=True, nu=3, omega_jac=0.8, gmres_m=30,
                          tol=1e-6, n_src=1, precision="mixed", seed=1, boundary="sponge")


ROWS = np.loadtxt(os.path.join(GOLDEN, "table6_constant_sponge.txt"), dtype=int)


@pytest.mark.parametrize("size,exact,w3,w4,w5", [tuple(r) for r in ROWS])
def test_table6_sponge_iterations(size, exact, w3, w4, w5):
    """Same bound as the PML block: never more than the printed count plus
    max(2, 25 %), and as many within that bound up to 1024^2.  At 2048^2 the
    printed counts rise (10 / 7 / 7) where this implementation's stay flat
    (6 at w = 3), so only the upper bound applies there."""
    hz = _hz()
    for (w, s_dd), paper in zip(((3, 15.0), (4, 20.0), (5, 25.0)), (w3, w4, w5)):
        cfg = _table6_sponge(int(size), w, s_dd)
        sv = hz.Solver.from_workload(cfg)
        sv.factor()
        _, st = sv.solve(torch.from_numpy(synth.sources(cfg)[0]).cuda())
        sv.close()
        assert st["relres_max"] <= cfg.tol
        tol = max(2, 0.25 * paper)
        assert st["iters_max"] <= paper + tol, (size, w, st["iters_max"], paper)
        if size <= 1024:
            assert abs(st["iters_max"] - paper) <= tol, (size, w, st["iters_max"], paper)
