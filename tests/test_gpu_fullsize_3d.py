"""The 3-D workloads at the size the benchmark runs them (64^3 interior cells
plus 12-cell PML: 87^3 = 658,503 unknowns per right-hand side).

* Configuration 4 recipe (layered medium, J = 12, X-sweep, mixed, 32 point
  sources in one call): every solution's true relative residual, computed
  with the oracle's assembled operator (Eq. 40 in 3-D), is below the GMRES
  tolerance 1e-6; this holds at any size and does not need the oracle's
  solves.
* Configuration 5 recipe (two-grid, gradient): the device gradient agrees
  with a central finite difference of the device misfit along a seeded
  direction (solves to 1e-10), and the misfit vanishes at the true model.
"""

import numpy as np
import pytest

import synth
from oracle import fd, mesh

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N3D = 64


def _hz():
    import paper_1412_0464_gb300 as hz
    hz.build()
    return hz


def test_config4_bench_size_32_sources_residuals():
    hz = _hz()
    cfg = synth.scaled_workload(4, N3D)
    assert cfg.n_src == 32 and cfg.shape == (87, 87, 87)
    m = synth.medium(cfg)
    s = hz.Solver.from_workload(cfg, m=m)
    s.factor()
    b = synth.sources(cfg)
    u, st = s.solve(torch.from_numpy(b).cuda())
    u = u.cpu().numpy()
    assert st["n_rhs"] == 32 and st["relres_max"] <= cfg.tol
    # the oracle's operator (same c_pml reading: mean wave speed over the unknowns)
    c_pml = float(np.mean(1.0 / np.sqrt(m)))
    axes = [mesh.fine_axis(c + 2 * cfg.w_out, cfg.w_out, cfg.h, cfg.s_out, c_pml)
            for c in cfg.cells]
    A = fd.assemble(axes, cfg.omega ** 2 * m, cfg.omega).tocsr()
    for r in range(32):
        br = b[r].ravel()
        res = np.linalg.norm(br - A @ u[r].ravel()) / np.linalg.norm(br)
        assert res <= 1.05 * cfg.tol, (r, res)


def test_config5_bench_size_gradient_directional_derivative():
    hz = _hz()
    cfg = synth.scaled_workload(5, N3D)
    m_true, m0 = synth.medium(cfg, "true"), synth.medium(cfg, "start")
    c_pml = float(np.mean(1.0 / np.sqrt(m0)))
    src = np.array([np.ravel_multi_index(tuple(int(v) for v in idx), cfg.shape)
                    for idx in synth.source_nodes(cfg)])
    rec = synth.receivers(cfg)
    s = hz.Solver.from_workload(cfg, m=m_true, c_pml=c_pml, tol=1e-10)
    s.factor()
    u, _ = s.solve(torch.from_numpy(synth.sources(cfg)).cuda())
    d = u.reshape(cfg.n_src, -1)[:, torch.from_numpy(rec).cuda()].cpu().numpy()
    phi_true, _, _ = s.grad(src, rec, d)
    assert phi_true <= 1e-16 * np.sum(np.abs(d) ** 2)

    def phi_at(m):
        s.set_medium(m)
        s.factor()
        return s.grad(src, rec, d)

    phi0, g0, st = phi_at(m0)
    assert st["relres_max"] <= 1e-10
    g0 = g0.cpu().numpy()
    dm = np.random.default_rng(55).standard_normal(m0.shape) * m0
    eps = 1e-4
    fp = phi_at(m0 + eps * dm)[0]
    fm = phi_at(m0 - eps * dm)[0]
    fdd = (fp - fm) / (2 * eps)
    an = float(np.sum(g0 * dm))
    assert abs(fdd - an) <= 1e-3 * abs(an), (fdd, an)
