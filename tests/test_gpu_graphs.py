"""The preconditioner application inside GMRES replays a captured CUDA graph
(one per input / output / right-hand-side count).  The replay runs the same
kernels in the same order, so the solution is bit-identical to uncaptured
launches (HZ_TEST_NO_GRAPH=1) for the X-sweep (two streams joined in the
graph), the UD-sweep and the two-grid cycle, in 2-D and 3-D; after a new
medium (levels rebuilt, graphs dropped) the solve is again correct."""

import numpy as np
import pytest

import synth
from oracle.problem import Problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _hz():
    import paper_1412_0464_gb300 as hz
    hz.build()
    return hz


@pytest.mark.parametrize("idx,n,w_out,J,sweep", [(2, 120, 8, 6, "X"), (2, 120, 8, 5, "UD"),
                                                  (3, 160, 8, 6, "X"), (4, 16, 4, 2, "X")])
def test_graph_replay_is_bit_identical(idx, n, w_out, J, sweep, monkeypatch):
    hz = _hz()
    cfg = synth.scaled_workload(idx, n, w_out=w_out, J=J, n_src=3)
    b = torch.from_numpy(synth.sources(cfg)[:3]).cuda()
    out = {}
    for mode in ("graph", "plain"):
        if mode == "plain":
            monkeypatch.setenv("HZ_TEST_NO_GRAPH", "1")
        s = hz.Solver.from_workload(cfg, sweep=sweep, max_rhs=3)
        s.factor()
        u1, st1 = s.solve(b)          # first solve: warm-up call, then captures
        u2, st2 = s.solve(b)          # second solve: replays
        out[mode] = (u2.cpu().numpy(), st2["iters_max"])
        assert torch.equal(u1, u2) and st1["iters_max"] == st2["iters_max"]
        s.close()
    assert np.array_equal(out["graph"][0], out["plain"][0])
    assert out["graph"][1] == out["plain"][1]


def test_graphs_dropped_on_new_medium():
    hz = _hz()
    cfg = synth.scaled_workload(2, 100, w_out=8, J=4, n_src=1)
    m1 = synth.medium(cfg)
    m2 = 1.0 / (1.0 / np.sqrt(m1) * 1.1) ** 2
    s = hz.Solver.from_workload(cfg, m=m1)
    b = torch.from_numpy(synth.sources(cfg)[0]).cuda()
    s.factor()
    s.solve(b)
    s.solve(b)
    s.set_medium(m2)
    s.factor()
    u, st = s.solve(b)
    A = Problem(cfg, m=m2).A
    bb = synth.sources(cfg)[0].ravel()
    res = np.linalg.norm(bb - A @ u.cpu().numpy().ravel()) / np.linalg.norm(bb)
    assert res <= 1.05 * cfg.tol
