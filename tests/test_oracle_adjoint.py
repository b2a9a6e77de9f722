"""Pins of the oracle's adjoint gradient (oracle/adjoint.py) to mathematics:
central finite differences of the misfit (directional and per node), the
zero gradient at the true model, and the complex symmetry of A that lets the
adjoint solve reuse A; with sponge layers (k^2 = omega^2 m (1 + i beta)^2,
Section 2.1) the finite differences also pin the sponge factor in dA/dm."""

import dataclasses

import numpy as np
import pytest

import synth
from oracle import adjoint, problem

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def _setup(n=32, boundary="pml"):
    cfg = dataclasses.replace(synth.adjoint_workload_2d(n), boundary=boundary)
    m_true = synth.medium(cfg, "true")
    m0 = synth.medium(cfg, "start")
    c_pml = float(np.mean(1.0 / np.sqrt(m0)))
    src = np.array([int(i) * cfg.N + int(j) for i, j in synth.source_nodes(cfg)])
    rec = synth.receivers(cfg)
    p_true = problem.Problem(cfg, m_true, two_grid=False, c_pml=c_pml)
    d = adjoint.synthetic_data(p_true, src, rec)
    return cfg, m_true, m0, c_pml, src, rec, d


def _phi(cfg, m, c_pml, src, rec, d):
    p = problem.Problem(cfg, m, two_grid=False, c_pml=c_pml)
    return adjoint.misfit_and_gradient(p, src, rec, d)[0]


def test_geometry():
    cfg = synth.adjoint_workload_2d(32)
    src = synth.source_nodes(cfg)
    rec = synth.receivers(cfg)
    assert src.shape == (8, 2) and rec.shape == (16,)
    assert len(set(src[:, 1])) == 8
    assert np.all(rec // cfg.N == cfg.w_out + 2)
    assert np.all(np.diff(rec) > 0)


def test_zero_at_true_model():
    cfg, m_true, m0, c_pml, src, rec, d = _setup()
    p = problem.Problem(cfg, m_true, two_grid=False, c_pml=c_pml)
    phi, g, _ = adjoint.misfit_and_gradient(p, src, rec, d)
    assert phi < 1e-25
    assert np.abs(g).max() < 1e-10


@pytest.mark.parametrize("boundary", ["pml", "sponge"])
def test_directional_finite_difference(boundary):
    cfg, m_true, m0, c_pml, src, rec, d = _setup(boundary=boundary)
    p = problem.Problem(cfg, m0, two_grid=False, c_pml=c_pml)
    phi, g, _ = adjoint.misfit_and_gradient(p, src, rec, d)
    assert phi > 0
    rng = np.random.default_rng(3)
    for _ in range(2):
        dm = rng.standard_normal(m0.shape) * m0
        eps = 1e-6
        fd = (_phi(cfg, m0 + eps * dm, c_pml, src, rec, d)
              - _phi(cfg, m0 - eps * dm, c_pml, src, rec, d)) / (2 * eps)
        an = float(np.sum(g * dm))
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-12 * phi, (fd, an)


@pytest.mark.parametrize("boundary", ["pml", "sponge"])
def test_per_node_finite_difference(boundary):
    """Brute force: the partial derivative at single nodes, including one in
    the outer PML (or sponge), one at a source and one at a receiver."""
    cfg, m_true, m0, c_pml, src, rec, d = _setup(boundary=boundary)
    p = problem.Problem(cfg, m0, two_grid=False, c_pml=c_pml)
    phi, g, _ = adjoint.misfit_and_gradient(p, src, rec, d)
    nodes = [int(src[3]), int(rec[5]), 2 * cfg.N + 3, (cfg.N // 2) * cfg.N + cfg.N // 2]
    for node in nodes:
        e = np.zeros(m0.size)
        e[node] = m0.ravel()[node]
        e = e.reshape(m0.shape)
        eps = 1e-5
        fd = (_phi(cfg, m0 + eps * e, c_pml, src, rec, d)
              - _phi(cfg, m0 - eps * e, c_pml, src, rec, d)) / (2 * eps)
        an = g.ravel()[node] * m0.ravel()[node]
        assert abs(fd - an) <= 1e-5 * abs(an) + 1e-9 * phi, (node, fd, an)


def test_dropped_conjugate_fails_fd():
    """A plausible slip (adjoint right-hand side without the conjugate)
    breaks the directional derivative."""
    cfg, m_true, m0, c_pml, src, rec, d = _setup()
    p = problem.Problem(cfg, m0, two_grid=False, c_pml=c_pml)
    import scipy.sparse.linalg as spla
    lu = spla.splu(p.A.tocsc())
    from oracle import fd as ofd
    w = ofd.rhs_scaling(p.axes, p.omega).ravel()
    g_bad = np.zeros(m0.size)
    for s, node in enumerate(src):
        b = np.zeros(m0.size, complex)
        b[node] = 1
        u = lu.solve(b)
        a = np.zeros(m0.size, complex)
        np.add.at(a, rec, u[rec] - d[s])
        g_bad += p.omega ** 2 * np.real(w * lu.solve(a) * u)
    _, g, _ = adjoint.misfit_and_gradient(p, src, rec, d)
    assert np.abs(g_bad - g.ravel()).max() > 1e-3 * np.abs(g).max()


def test_complex_symmetric():
    cfg = synth.adjoint_workload_2d(32)
    p = problem.Problem(cfg, synth.medium(cfg, "start"), two_grid=False)
    A = p.A.tocsr()
    assert abs(A - A.T).max() == 0
    assert abs(A - A.conj().T).max() > 0
