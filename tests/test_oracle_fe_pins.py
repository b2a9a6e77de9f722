"""Pins of the coarse level's PML rows and its k^2 averaging (Appendix A.2-A.3).

* Coarse k^2 (Appendix A.3, last paragraph): the 1-D weights (1/2, 1/2) on an
  unrefined coarse cell and (1/4, 1/2, 1/4) on a refined one are exactly the
  cell mean of the piecewise-linear interpolant of the fine nodal values, so
  the tensor averaging must equal the mean of the multilinear interpolant
  over every coarse cell.  The mean is computed here by Gauss quadrature of
  the interpolant (scipy's RegularGridInterpolator), with non-polynomial
  fields that tell the weights apart.
* FE operator with PML (Eqs. 53-61): with the coefficients of exactly
  integrated multilinear elements (c = 4/9, 4/9, 2/3 in 2-D; 8/27, 4/9, 2/9,
  4/9, 4/9 in 3-D) the cell sum must equal the Galerkin matrix of the
  PML-stretched operator
      a(u, v) = sum_cells int  sum_l (alpha_l / prod_{m != l} alpha_m) u_l v_l
                             - k^2 / prod_m alpha_m u v,
  with alpha, h and k^2 constant per cell (alpha at the cell midpoints), on
  the PML-aware coarse mesh (PML cells of size h, interior cells 2h).  The
  Galerkin integrals are evaluated here by 2-point Gauss quadrature of the
  multilinear shape functions, independently of the I_a / J_b constants.
* Planted mistakes (swapped averaging weights, thirds, alpha/h <-> h/alpha,
  alpha sampled at the cell's left node) fail these pins.
"""

import itertools

import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

from oracle import fe, mesh

GAUSS = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))   # on [0, 1], weights 1/2


def _coarse(dim, n_int=12, w=3, h=1.0 / 24):
    co = [mesh.coarse_axis(n_int, w, h, 20.0, 1.3) for _ in range(dim)]
    return co, n_int + 2 * w


def _quadrature_cell_means(kp, i_fp, h):
    """Mean of the multilinear interpolant of the padded nodal field kp (fine
    nodes 0..n_cells on every axis, node p at x = p h) over every coarse cell."""
    d = kp.ndim
    nodes = np.arange(kp.shape[0]) * h
    interp = RegularGridInterpolator([nodes] * d, kp, method="linear")
    n_c = i_fp.size - 1
    out = np.zeros((n_c,) * d)
    for c in itertools.product(range(n_c), repeat=d):
        # fine cells inside the coarse cell, per axis
        spans = [range(i_fp[c[l]], i_fp[c[l] + 1]) for l in range(d)]
        acc, vol = 0.0, 1.0
        for l in range(d):
            vol *= (i_fp[c[l] + 1] - i_fp[c[l]]) * h
        for fc in itertools.product(*spans):
            pts = np.array([[(fc[l] + g[l]) * h for l in range(d)]
                            for g in itertools.product(GAUSS, repeat=d)])
            acc += interp(pts).sum() * (0.5 ** d) * h ** d
        out[c] = acc / vol
    return out


def _k2_field(shape, seed):
    """Non-polynomial nodal field: smooth part plus noise (tells weights apart)."""
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[np.linspace(0, 1, s) for s in shape], indexing="ij")
    smooth = 40.0 + 10.0 * np.sin(3.0 * sum(grids)) + 5.0 * np.exp(grids[-1] * 2.0)
    return smooth * (1.0 + 0.3 * rng.random(shape))


def _k2_error(dim, seed=0):
    co, n_cells = _coarse(dim, n_int=8 if dim == 3 else 12, w=2 if dim == 3 else 3)
    i_fp, refined = co[0][1], co[0][2]
    h = 1.0 / 24
    N = n_cells - 1
    k2 = _k2_field((N,) * dim, seed)
    got = fe.coarse_k2(k2, i_fp, refined)
    want = _quadrature_cell_means(np.pad(k2, 1, mode="edge"), i_fp, h)
    return np.abs(got - want).max() / np.abs(want).max()


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_coarse_k2_is_cell_mean_of_multilinear_interpolant(dim):
    assert _k2_error(dim) < 1e-13


@pytest.mark.parametrize("weights", ["swapped", "thirds", "midpoint"])
def test_planted_averaging_mistakes_fail_the_k2_pin(weights, monkeypatch):
    real = fe.averaging_1d

    def planted(i_fp, refined, n_fine_cells):
        W = real(i_fp, refined, n_fine_cells)
        for Q in range(refined.size):
            p = i_fp[Q]
            if weights == "swapped":          # refined and unrefined rules exchanged
                W[Q, :] = 0
                if refined[Q]:
                    W[Q, p:p + 2] = (0.5, 0.5)
                else:
                    q = min(p, W.shape[1] - 3)
                    W[Q, q:q + 3] = (0.25, 0.5, 0.25)
            elif weights == "thirds" and refined[Q]:
                W[Q, p:p + 3] = (1 / 3, 1 / 3, 1 / 3)
            elif weights == "midpoint" and refined[Q]:
                W[Q, p:p + 3] = (0.0, 1.0, 0.0)
        return W

    monkeypatch.setattr(fe, "averaging_1d", planted)
    assert _k2_error(2) > 1e-3


# --------------------------------------------------------------- FE with PML
Q1_COEFFS = {2: (4 / 9, 4 / 9, 2 / 3), 3: (8 / 27, 4 / 9, 2 / 9, 4 / 9, 4 / 9)}


def _alpha(sigma, omega):
    return 1.0 / (1.0 + 1j * sigma / omega)


def _galerkin(axes, k2cell, omega):
    """Q1 Galerkin matrix of the PML-stretched operator by Gauss quadrature."""
    d = len(axes)
    Ns = [ax.N for ax in axes]
    n = int(np.prod(Ns))
    A = np.zeros((n, n), dtype=np.complex128)
    pts = list(itertools.product(GAUSS, repeat=d))

    def phi(a, xi):
        return np.prod([xi[l] if a[l] else 1.0 - xi[l] for l in range(d)])

    def dphi(a, xi, l, hl):       # d/dx_l of the shape function of corner a
        v = (1.0 if a[l] else -1.0) / hl
        for m in range(d):
            if m != l:
                v *= xi[m] if a[m] else 1.0 - xi[m]
        return v

    for c in itertools.product(*[range(N + 1) for N in Ns]):
        hl = [axes[l].h_cell[c[l]] for l in range(d)]
        al = [_alpha(axes[l].sigma_cell[c[l]], omega) for l in range(d)]
        vol, pa = np.prod(hl), np.prod(al)
        k2 = k2cell[c]
        corners = list(itertools.product((0, 1), repeat=d))
        for a in corners:
            ia = [c[l] + a[l] - 1 for l in range(d)]
            if any(x < 0 or x >= Ns[l] for l, x in enumerate(ia)):
                continue
            ra = np.ravel_multi_index(ia, Ns)
            for b in corners:
                ib = [c[l] + b[l] - 1 for l in range(d)]
                if any(x < 0 or x >= Ns[l] for l, x in enumerate(ib)):
                    continue
                rb = np.ravel_multi_index(ib, Ns)
                val = 0.0
                for xi in pts:
                    wq = 0.5 ** d * vol
                    stiff = sum(al[l] * al[l] / pa * dphi(a, xi, l, hl[l]) * dphi(b, xi, l, hl[l])
                                for l in range(d))
                    val += wq * (stiff - k2 / pa * phi(a, xi) * phi(b, xi))
                A[ra, rb] += val
    return A


def _fe_case(dim):
    n_int, w = (8, 3) if dim == 2 else (4, 2)
    h = 1.0 / (2 * n_int)
    omega = 23.0
    co = [mesh.coarse_axis(n_int, w, h, 30.0, 1.7) for _ in range(dim)]
    axes = [c[0] for c in co]
    rng = np.random.default_rng(11)
    k2cell = omega ** 2 * (0.3 + rng.random(tuple(a.N + 1 for a in axes)))
    return axes, k2cell, omega, 2 * h


def _fe_error(dim):
    axes, k2cell, omega, H = _fe_case(dim)
    got = fe.assemble(axes, k2cell, omega, H, coeffs=Q1_COEFFS[dim]).toarray()
    want = _galerkin(axes, k2cell, omega)
    return np.abs(got - want).max() / np.abs(want).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_fe_with_pml_equals_q1_galerkin(dim):
    axes, _, omega, _ = _fe_case(dim)
    # the case really has PML cells of both sizes and complex alpha
    assert np.any(axes[0].sigma_cell > 0) and len(set(np.round(axes[0].h_cell, 12))) == 2
    assert _fe_error(dim) < 1e-13


@pytest.mark.parametrize("flaw", ["alpha_over_h_swapped", "alpha_at_left_node"])
def test_planted_pml_mistakes_fail_the_galerkin_pin(flaw, monkeypatch):
    if flaw == "alpha_over_h_swapped":
        monkeypatch.setattr(fe, "_stiff_factor", lambda a, h: h / a)
        monkeypatch.setattr(fe, "_other_factor", lambda a, h: a / h)
    else:
        def left_node(self, omega):
            s = np.concatenate([[0.0], self.sigma_node])    # sigma at the cell's left node
            return 1.0 / (1.0 + 1j * s / omega)
        monkeypatch.setattr(mesh.Axis, "alpha_cell", left_node)
    assert _fe_error(2) > 1e-3
