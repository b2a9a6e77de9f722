"""Pins of the sponge boundary layer and the standard two-grid cycle (Sections 2.1, 4.1).

* Sponge profile: beta = beta_max (d / L)^2 with the one-way amplitude damping
  exp(-int k beta dx) = exp(-k beta_max L / 3) set to the requested factor
  (exact integral of the quadratic profile, checked by quadrature).
* 1-D point source in a constant medium with sponge layers: the field inside
  agrees with the closed-form discrete free-space Green's function (the
  sponge absorbs; its reflection shrinks as the layer widens), and inside the
  layer it decays by about the set factor; a sign slip (k (1 - i beta), an
  amplifying layer) breaks the agreement.
* The operator is complex symmetric and equals the plain Eq. 40 rows inside.
* Standard coarsening (all cells merged in pairs): the coarse axis has no
  kept cells, cells of size 2h, and P reproduces linear functions.
* Table 6 of the paper, "Constant medium, sponge" block, 256^2: TGSP needs
  5 iterations for w = 3, 4, 5 (printed: 5, 5, 5); the sponge needs fewer
  iterations than the PML (printed: 10).
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spla
from scipy.integrate import quad

import synth
from oracle import fd, fe, mesh
from oracle.problem import Problem


def test_sponge_beta_max_gives_the_damping():
    k, L, D = 2 * np.pi * 10.0, 0.08, 1e-2
    bmax = mesh.sponge_beta_max(D, k, L)
    integral, _ = quad(lambda x: k * bmax * (x / L) ** 2, 0.0, L)
    assert np.exp(-integral) == pytest.approx(D, rel=1e-12)


def _sponge_1d(n=400, w=80, k=2 * np.pi * 10.0, D=1e-2, sign=+1.0):
    h = 1.0 / n
    ax = mesh.fine_axis(n + 2 * w, w, h, 0.0, 1.0)          # no PML
    beta = mesh.sponge_beta(n + 2 * w, w, h, mesh.sponge_beta_max(D, k, w * h))
    k2 = k * k * (1.0 + sign * 1j * beta) ** 2
    A = fd.assemble([ax], k2, k)
    s = ax.N // 2
    b = np.zeros(ax.N, complex)
    b[s] = 1.0
    u = spla.spsolve(A.tocsc(), b)
    t = np.arccos(1 - (k * h) ** 2 / 2)
    jj = np.arange(ax.N)
    exact = 1j * h / (2 * np.sin(t)) * np.exp(1j * t * np.abs(jj - s))
    inner = (jj >= w) & (jj < ax.N - w)
    err = np.abs(u[inner] - exact[inner]).max() / np.abs(exact).max()
    return u, exact, err, w, s


def test_sponge_1d_matches_free_space_and_decays():
    errs = [_sponge_1d(w=w)[2] for w in (20, 40, 80)]
    assert errs[-1] < 2e-2                    # several wavelengths: small reflection
    assert errs[0] > errs[-1]
    u, exact, _, w, s = _sponge_1d(w=80)
    # amplitude through the layer (outer edge vs inner edge), about the set factor
    ratio = abs(u[-2]) / abs(u[-w])
    assert 1e-3 < ratio < 1e-1


def test_planted_amplifying_sponge_fails():
    assert _sponge_1d(w=80, sign=-1.0)[2] > 1e-1


def test_sponge_operator_symmetric_and_plain_inside():
    cfg = synth.scaled_workload(2, 40, w_out=10, J=4, boundary="sponge")
    p = Problem(cfg)
    assert abs(p.A - p.A.T).max() == 0.0
    q = Problem(synth.scaled_workload(2, 40, w_out=10, J=4, s_out=0.0), m=p.m)
    c = (cfg.shape[0] // 2) * cfg.shape[1] + cfg.shape[1] // 2     # an interior row
    assert abs(p.A[c] - q.A[c]).max() == 0.0
    assert np.iscomplexobj(p.k2) and np.abs(p.k2.imag).max() > 0


def test_standard_coarsening_axis():
    n_all, h = 60, 1.0 / 40
    ax, i_fp, refined = mesh.coarse_axis(n_all, 0, h, 0.0, 1.0)
    assert np.all(refined) and np.allclose(ax.h_cell, 2 * h)
    assert np.all(np.diff(i_fp) == 2)
    N = n_all - 1
    P = fe.prolongation_1d(i_fp, refined, N)
    xc, xf = i_fp[1:-1] * h, np.arange(1, N + 1) * h
    got = P @ (0.3 + 2.0 * xc)
    inner = (xf > i_fp[1] * h) & (xf < i_fp[-2] * h)
    assert np.abs(got[inner] - (0.3 + 2.0 * xf[inner])).max() < 1e-13


def _table6_sponge(n, w, s, boundary):
    cells = n // 2 + 2 * 18
    J = cells // (2 * w + 1)
    J -= J % 2
    return synth.Workload(name="table6s", dim=2, n=n, w_out=36 if boundary == "sponge" else 4,
                          ppw=10.0, c_min=1.0, medium="const", corr=0.0, J=J, w_dd=w, s_dd=s,
                          s_out=20.0, sweep="UD", two_grid=True, nu=3, omega_jac=0.8,
                          gmres_m=30, tol=1e-6, n_src=1, precision="fp64", seed=1,
                          boundary=boundary)


@pytest.mark.slow
def test_table6_sponge_rows_256():
    its = {}
    for w, s in ((3, 15.0), (4, 20.0), (5, 25.0)):
        cfg = _table6_sponge(256, w, s, "sponge")
        _, info = Problem(cfg).solve(synth.sources(cfg)[0])
        assert info["converged"]
        its[w] = info["iters"]
        assert abs(its[w] - 5) <= 2, (w, its[w])
    cfg = _table6_sponge(256, 4, 20.0, "pml")
    _, info = Problem(cfg).solve(synth.sources(cfg)[0])
    assert its[4] < info["iters"]
