"""The paper's constant-medium regression tables, run through hz_solve on the GPU.

* Table 6, "Constant medium, PML" block (tests/golden/table6_constant_pml.txt):
  TGSP (Section 4) iterations to a 1e-6 residual reduction at 10 points per
  wavelength for 256^2 .. 2048^2 and DD PML widths w = 3, 4, 5 (S_pml =
  15 / 20 / 25), nu = 3, omega_Jac = 0.8, outer PML 4 cells, UD-sweeps on
  floor(N_x / (2 w + 1)) coarse slabs (made even).  The media and sizes are
  the paper's; the iteration count may differ by the discretisation readings,
  so the bound is max(2, 25 %) of the printed count.  (The "exact coarse
  solve" column needs one slab spanning the coarse grid, wider than the 2-D
  slab kernels take; the oracle reproduces it at 256^2.)
* Table 4 (sweep patterns, constant medium 2048^2): the X-sweep needs the
  same number of iterations as the UD-sweep (within one), the partial
  NX-sweeps more.
"""

import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hz():
    import paper_1412_0464_gb300 as hz
    hz.build()
    return hz


def _table6_workload(n, w, s, sweep="UD"):
    cells = n // 2 + 2 * 4
    J = cells // (2 * w + 1)
    J -= J % 2
    return synth.Workload(name="table6", dim=2, n=n, w_out=4, ppw=10.0, c_min=1.0,
                          medium="const", corr=0.0, J=J, w_dd=w, s_dd=s, s_out=20.0,
                          sweep=sweep, two_grid=True, nu=3, omega_jac=0.8, gmres_m=30,
                          tol=1e-6, n_src=1, precision="mixed", seed=1)


def _iters(hz, cfg, **over):
    s = hz.Solver.from_workload(cfg, **over)
    s.factor()
    _, st = s.solve(torch.from_numpy(synth.sources(cfg)[0]).cuda())
    s.close()
    assert st["relres_max"] <= cfg.tol
    return st["iters_max"]


ROWS = np.loadtxt(os.path.join(GOLDEN, "table6_constant_pml.txt"), dtype=int)


@pytest.mark.parametrize("size,exact,w3,w4,w5", [tuple(r) for r in ROWS])
def test_table6_tgsp_iterations(size, exact, w3, w4, w5):
    """Never more than the printed count (plus the bound); as many (within the
    bound) where the printed counts stay flat (<= 15).  The printed 32 at
    2048^2, w = 3 -- the paper's case of a DD PML too thin for the size -- is
    the one entry this implementation beats by far (12 iterations)."""
    hz = _hz()
    got = {}
    for (w, s), paper in zip(((3, 15.0), (4, 20.0), (5, 25.0)), (w3, w4, w5)):
        got[w] = _iters(hz, _table6_workload(int(size), w, s))
        tol = max(2, 0.25 * paper)
        assert got[w] <= paper + tol, (size, w, got[w], paper)
        if paper <= 15:
            assert abs(got[w] - paper) <= tol, (size, w, got[w], paper)


def test_table4_sweep_patterns():
    hz = _hz()
    cfg = _table6_workload(2048, 4, 20.0)
    its = {sw: _iters(hz, cfg, sweep=sw) for sw in ("UD", "X")}
    its["NX2"] = _iters(hz, cfg, sweep="NX", n_cell=2)
    assert abs(its["UD"] - its["X"]) <= 1, its
    assert its["NX2"] > its["X"], its
