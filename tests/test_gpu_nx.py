"""The NX-sweep (SweepingPrecNX, Table 3, partial sweeps) on the GPU against the oracle.

One application element by element (FP64 1e-9, complex64 3e-4, as for the
other sweeps), the one-cell case equal to the X-sweep, and the ordering of
Table 7 (the partial sweeps need more GMRES iterations than the X-sweep).
"""

import numpy as np
import pytest

import synth
from oracle.problem import Problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-9, "mixed": 3e-4}


def _hz():
    import paper_1412_0464_gb300 as hz
    hz.build()
    return hz


def _close(a, b, tol):
    rel = np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())
    return rel <= tol and np.abs(a - b).max() <= tol * np.abs(b).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("idx,n,w_out,J,n_cell", [(2, 101, 7, 7, 2), (2, 120, 8, 9, 3),
                                                   (3, 96, 6, 6, 2), (4, 16, 4, 5, 2)])
def test_nx_preconditioner_matches_oracle(idx, n, w_out, J, n_cell, precision):
    hz = _hz()
    cfg = synth.scaled_workload(idx, n, w_out=w_out, J=J, n_src=2)
    p = Problem(cfg, sweep="NX", n_cell=n_cell)
    s = hz.Solver.from_workload(cfg, precision=precision, sweep="NX", n_cell=n_cell)
    s.factor()
    f = np.random.default_rng(8).standard_normal((2,) + cfg.shape) + 0.3j
    z = s.precond(torch.from_numpy(f).cuda()).cpu().numpy()
    for r in range(2):
        assert _close(z[r], p.precondition(f[r]).reshape(cfg.shape), TOL[precision])


def test_nx_one_cell_is_the_x_sweep():
    hz = _hz()
    cfg = synth.scaled_workload(2, 90, w_out=8, J=6)
    f = torch.from_numpy(np.random.default_rng(9).standard_normal(cfg.shape) + 0j).cuda()
    zx = hz.Solver.from_workload(cfg, precision="fp64", sweep="X")
    zx.factor()
    z1 = hz.Solver.from_workload(cfg, precision="fp64", sweep="NX", n_cell=1)
    z1.factor()
    a, b = zx.precond(f).cpu().numpy(), z1.precond(f).cpu().numpy()
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_table7_ordering_on_gpu():
    """Constant medium (configuration 1 recipe), J = 16: the X-sweep needs fewer
    iterations than every partial sweep, NX(2) no more than NX(8)."""
    hz = _hz()
    cfg = synth.scaled_workload(1, 400, w_out=10, J=16)
    b = torch.from_numpy(synth.sources(cfg)[0]).cuda()
    its = []
    for sweep, nc in (("X", 1), ("NX", 2), ("NX", 4), ("NX", 8)):
        s = hz.Solver.from_workload(cfg, precision="mixed", sweep=sweep, n_cell=nc)
        s.factor()
        _, st = s.solve(b)
        assert st["relres_max"] <= cfg.tol
        its.append(st["iters_max"])
        s.close()
    assert its[0] < min(its[1:]) and its[1] <= its[3], its
