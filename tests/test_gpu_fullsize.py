"""Parity at the full sizes the benchmark runs, on the paths those sizes select.

Configuration 2 (1039^2 unknowns, J = 16, slab width W = 72..74): the slab
kernels' W <= 80 tile templates, the automatic segment count (two segment
CTAs per SM in complex64) and its two-level carries; configuration 3
(4059^2 fine unknowns, coarse FE level 2059^2, J = 32 coarse slabs, W ~ 73,
automatic P = 304).  Slab solves and one preconditioner application are
compared element by element with the FP64 oracle (SuperLU slab solves,
Tables 2-3); the full solves are checked through the oracle's assembled
operator (true relative residual) and against the plain-FP64 GPU arm.
"""

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


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def _close(a, b, tol):
    return _rel(a, b) <= tol and np.abs(a - b).max() <= tol * np.abs(b).max()


TOL = {"fp64": 1e-9, "mixed": 3e-4}


@pytest.fixture(scope="module")
def c2():
    cfg = synth.workload(2)
    return cfg, Problem(cfg)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_config2_slab_solves_at_full_width(c2, precision):
    hz = _hz()
    cfg, p = c2
    s = hz.Solver.from_workload(cfg, m=p.m, precision=precision, max_rhs=2)
    s.factor()
    widths = []
    for j in (1, 2, 8, 9, 15, 16):
        sl = p.dd.slabs[j]
        info = s.slab_info(j)
        assert (info["lo"], info["hi"], info["wl"], info["wr"], info["W"]) == \
            (sl.lo, sl.hi, sl.wl, sl.wr, sl.W)
        widths.append(sl.W)
        fd = _rand((2, cfg.N, sl.W), 100 + j)
        ud = s.slab_solve(j, torch.from_numpy(fd).cuda()).cpu().numpy()
        for r in range(2):
            ref = sl.lu.solve(fd[r].ravel()).reshape(cfg.N, sl.W)
            assert _close(ud[r], ref, TOL[precision]), (j, r, _rel(ud[r], ref))
    assert min(widths) >= 65 and max(widths) <= 80      # the W <= 80 templates
    s.close()


def test_config2_preconditioner_at_full_size(c2):
    hz = _hz()
    cfg, p = c2
    s = hz.Solver.from_workload(cfg, m=p.m, precision="mixed")
    s.factor()
    f = _rand(cfg.shape, 9)
    z = s.precond(torch.from_numpy(f).cuda()).cpu().numpy()
    ref = p.dd.apply(f, cfg.sweep)
    assert _close(z, ref, TOL["mixed"])
    s.close()


@pytest.fixture(scope="module")
def c3():
    """The parts of the configuration-3 oracle these tests need (the whole
    oracle, with all 32 coarse slab factorisations and its GMRES, is too slow
    for a test): the fine operator (Eq. 40) and four coarse slabs."""
    from oracle import dd, fd, fe, mesh
    cfg = synth.workload(3)
    m = synth.medium(cfg)
    c_pml = float(np.mean(1.0 / np.sqrt(m)))
    axes = [mesh.fine_axis(cfg.n_cells, cfg.w_out, cfg.h, cfg.s_out, c_pml) for _ in range(2)]
    A = fd.assemble(axes, cfg.omega ** 2 * m, cfg.omega)
    co = [mesh.coarse_axis(cfg.n, cfg.w_out, cfg.h, cfg.s_out, c_pml) for _ in range(2)]
    caxes = [c[0] for c in co]
    k2c = fe.coarse_k2(cfg.omega ** 2 * m, co[0][1], co[0][2])
    H, om = 2.0 * cfg.h, cfg.omega
    Ac = fe.assemble(caxes, k2c, om, H)
    slabs = dd.SweepingDD(caxes, k2c, "cell", lambda ax, med: fe.assemble(ax, med, om, H), Ac,
                          cfg.J, cfg.w_dd, cfg.s_dd, c_pml, om, only=(1, 16, 17, 32)).slabs

    class P:
        pass
    p = P()
    p.m, p.A, p.slabs = m, A, slabs
    return cfg, p


def test_config3_coarse_slab_solves_at_full_size(c3):
    hz = _hz()
    cfg, p = c3
    s = hz.Solver.from_workload(cfg, m=p.m, precision="mixed")
    s.factor()
    for j in (1, 16, 17, 32):
        sl = p.slabs[j]
        info = s.slab_info(j)
        assert info["W"] == sl.W
        nt = sl.A.shape[0] // sl.W
        fd = _rand((nt, sl.W), 200 + j)
        ud = s.slab_solve(j, torch.from_numpy(fd).cuda()).cpu().numpy()
        ref = sl.lu.solve(fd.ravel()).reshape(fd.shape)
        assert _close(ud, ref, TOL["mixed"]), (j, _rel(ud, ref))
    s.close()


def test_config3_full_solve(c3):
    hz = _hz()
    cfg, p = c3
    b = synth.sources(cfg)[0]
    out = {}
    for precision in ("mixed", "fp64"):
        s = hz.Solver.from_workload(cfg, m=p.m, precision=precision)
        s.factor()
        u, st = s.solve(torch.from_numpy(b).cuda())
        u = u.cpu().numpy()
        relres = np.linalg.norm(p.A @ u.ravel() - b.ravel()) / np.linalg.norm(b)
        assert st["relres_max"] <= cfg.tol and relres <= 1.05 * cfg.tol
        out[precision] = (u, st["iters_max"])
        s.close()
    assert abs(out["mixed"][1] - out["fp64"][1]) <= 1
    assert _rel(out["mixed"][0], out["fp64"][0]) <= 1e-5
