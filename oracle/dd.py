"""Double-sweep domain decomposition with PML transmission (Section 2).

Discrete formulation of Section 2.2.  The sweep axis is x, the last array
axis; columns are unknown indices 0..N-1 along x.

* Partition: beta_0 = -1, beta_J = N - 1 and an equal split in between
  (the first N mod J slabs one column wider); Eq. 17: tilde-beta_0 = beta_0,
  tilde-beta_J = beta_J, tilde-beta_j = beta_j - 1.  The forward interval
  ]b_{j-1}, b_j[ is the column set {beta_{j-1}+1 .. beta_j}.
* Subdomain (Eq. 9): the core is the columns tilde-beta_{j-1}+1 .. beta_j
  (since tilde-b_j < b_j); w PML columns are added on every internal side.
  The added PML starts at the interface half point (sigma = 0 there): the
  m-th added column is at distance (m - 1/2) h_I, the cell beyond it at
  (m - 1) h_I .. m h_I, with d_pml = w h_I (h_I the interface cell size).
* Frozen k (Eq. 10): in the added columns k equals k on the adjacent core
  boundary (nodal k for finite differences, the interface cell's k for the
  cellwise finite-element operator).
* A^(j): the same discretisation on the extended mesh.
* Transmission (Eqs. 19-20) uses the entries of the global A between the
  two layers.
* Algorithms: Table 2 (SubdomSolve, ForwardSweep, BackwardSweep,
  MidSolveIn, MidSolveOut) and Table 3 (SweepingPrecUD, SweepingPrecX).
  Transmission from or to a neighbour that does not exist is dropped
  (T^(1) = tilde-T^(J) = 0, Section 2.1).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .mesh import Axis


def partition(N: int, J: int):
    """beta_0..beta_J and tilde-beta_0..tilde-beta_J (Eq. 17)."""
    sizes = [N // J + (1 if j < N % J else 0) for j in range(J)]
    beta = [-1]
    for s in sizes:
        beta.append(beta[-1] + s)
    assert beta[-1] == N - 1
    beta_t = [beta[0]] + [b - 1 for b in beta[1:-1]] + [beta[-1]]
    return beta, beta_t


class Slab:
    """Subdomain Omega^(j): mesh, operator and factorisation."""

    def __init__(self, j, lo, hi, wl, wr, axis_x: Axis, medium, A):
        self.j, self.lo, self.hi, self.wl, self.wr = j, lo, hi, wl, wr
        self.axis_x = axis_x
        self.medium = medium
        self.W = axis_x.N
        self.A = A.tocsc()
        self.lu = spla.splu(self.A)

    def local(self, g: int) -> int:
        """Slab column of global column g."""
        return g - self.lo + self.wl


class SweepingDD:
    """The sweeping preconditioners P_UD and P_X of Table 3.

    ``builder(axes, medium)`` assembles the discretisation on a mesh;
    ``medium_kind`` is "node" (k^2 at unknowns, finite differences) or
    "cell" (k^2 per cell, finite elements).
    """

    def __init__(self, axes: list[Axis], medium: np.ndarray, medium_kind: str, builder,
                 A: sp.spmatrix, J: int, w: int, s_dd: float, c_pml: float, omega: float,
                 only=None):
        self.axes, self.medium, self.kind, self.builder = axes, medium, medium_kind, builder
        self.A = A.tocsr()
        self.J, self.w, self.s_dd, self.c_pml, self.omega = J, w, s_dd, c_pml, omega
        self.shape = tuple(ax.N for ax in axes)
        self.N = self.shape[-1]
        self.nt = int(np.prod(self.shape[:-1])) if len(self.shape) > 1 else 1
        self.beta, self.beta_t = partition(self.N, J)
        # ``only`` (tests at large sizes): build just these slabs; the sweeps
        # need all of them
        self.slabs = [None] + [self._make_slab(j) if only is None or j in only else None
                               for j in range(1, J + 1)]
        self._blocks = {}

    # ----------------------------------------------------------------- set-up
    def _dd_sigma(self, dist, h_I):
        C = self.s_dd * self.c_pml / (self.w * h_I) ** 3
        return C * dist * dist

    def _make_slab(self, j: int) -> Slab:
        gx = self.axes[-1]
        lo = self.beta_t[j - 1] + 1
        hi = self.beta[j]
        wl = self.w if j > 1 else 0
        wr = self.w if j < self.J else 0
        W = hi - lo + 1 + wl + wr
        hIl, hIr = gx.h_cell[lo], gx.h_cell[hi + 1]
        g = np.arange(W) - wl + lo                       # global column of each slab column
        sig_node = np.empty(W)
        for e in range(W):
            if g[e] < lo:
                sig_node[e] = self._dd_sigma((lo - g[e] - 0.5) * hIl, hIl)
            elif g[e] > hi:
                sig_node[e] = self._dd_sigma((g[e] - hi - 0.5) * hIr, hIr)
            else:
                sig_node[e] = gx.sigma_node[g[e]]
        gc = np.arange(W + 1) - wl + lo                  # global cell of each slab cell
        sig_cell = np.empty(W + 1)
        h_cell = np.empty(W + 1)
        for c in range(W + 1):
            if gc[c] < lo:
                sig_cell[c] = self._dd_sigma((lo - gc[c]) * hIl, hIl)
                h_cell[c] = hIl
            elif gc[c] > hi + 1:
                sig_cell[c] = self._dd_sigma((gc[c] - hi - 1) * hIr, hIr)
                h_cell[c] = hIr
            else:
                sig_cell[c] = gx.sigma_cell[gc[c]]
                h_cell[c] = gx.h_cell[gc[c]]
        axis = Axis(h_cell=h_cell, sigma_node=sig_node, sigma_cell=sig_cell)
        if self.kind == "node":
            med = self.medium[..., np.clip(g, lo, hi)]
        else:
            med = self.medium[..., np.clip(gc, lo, hi + 1)]
        A = self.builder(self.axes[:-1] + [axis], med)
        return Slab(j, lo, hi, wl, wr, axis, med, A)

    def _cols(self, x: int) -> np.ndarray:
        """Flat indices of all unknowns in global column x."""
        return np.arange(self.nt) * self.N + x

    def block(self, x1: int, x2: int):
        """Coupling block A_{x1, x2} of the global matrix between two columns."""
        key = (x1, x2)
        if key not in self._blocks:
            self._blocks[key] = self.A[self._cols(x1)][:, self._cols(x2)].tocsr()
        return self._blocks[key]

    # -------------------------------------------------------- Table 2 helpers
    def _T(self, j, B):
        """T^(j) B (Eq. 19) at the layers beta_{j-1}, beta_{j-1}+1."""
        b = self.beta[j - 1]
        return (self.block(b, b + 1) @ B[1], -(self.block(b + 1, b) @ B[0]))

    def _Tt(self, j, B):
        """tilde-T^(j) B (Eq. 20) at the layers tilde-beta_j, tilde-beta_j+1."""
        b = self.beta_t[j]
        return (-(self.block(b, b + 1) @ B[1]), self.block(b + 1, b) @ B[0])

    def subdom_solve(self, u, f, j, a, b, at, bt, tau1, B1, tau2, B2, tau3, B3, tau4, B4):
        """SubdomSolve of Table 2 (u, f: global fields, flattened to (nt, N))."""
        s = self.slabs[j]
        tau1 = tau1 and j > 1
        tau4 = tau4 and j > 1
        tau2 = tau2 and j < self.J
        tau3 = tau3 and j < self.J
        fd = np.zeros((self.nt, s.W), dtype=np.complex128)
        fd[:, s.local(a + 1):s.local(b) + 1] = f[:, a + 1:b + 1]          # J(j,a,b) f
        if tau1:
            t0, t1 = self._T(j, B1)
            x = self.beta[j - 1]
            fd[:, s.local(x)] += t0
            fd[:, s.local(x + 1)] += t1
        if tau3:
            t0, t1 = self._Tt(j, B3)
            x = self.beta_t[j]
            fd[:, s.local(x)] += t0
            fd[:, s.local(x + 1)] += t1
        ud = s.lu.solve(fd.ravel()).reshape(self.nt, s.W)                # (A^(j))^-1 f_d
        u[:, at + 1:bt + 1] += ud[:, s.local(at + 1):s.local(bt) + 1]    # J(j,at,bt)^T u_d
        if tau2:
            x = self.beta[j]
            B2[0], B2[1] = ud[:, s.local(x)].copy(), ud[:, s.local(x + 1)].copy()
        if tau4:
            x = self.beta_t[j - 1]
            B4[0], B4[1] = ud[:, s.local(x)].copy(), ud[:, s.local(x + 1)].copy()

    def forward_sweep(self, u, f, j0, j1, B):
        be = self.beta
        for j in range(j0, j1 + 1):
            self.subdom_solve(u, f, j, be[j - 1], be[j], be[j - 1], be[j],
                              j > 1, B, j < self.J, B, False, None, False, None)

    def backward_sweep(self, u, f, j0, j1, B):
        bt = self.beta_t
        for j in range(j0, j1 - 1, -1):
            self.subdom_solve(u, f, j, bt[j - 1], bt[j], bt[j - 1], bt[j],
                              False, None, False, None, j < self.J, B, j > 1, B)

    def mid_solve_in(self, u, f, j, B1, B2):
        be, bt = self.beta, self.beta_t
        self.subdom_solve(u, f, j, be[j - 1], bt[j], be[j - 1], bt[j],
                          True, B1, False, None, True, B2, False, None)

    def mid_solve_out(self, u, f, j, B1, B2):
        be, bt = self.beta, self.beta_t
        self.subdom_solve(u, f, j, bt[j - 1], be[j], bt[j - 1], be[j],
                          False, None, True, B1, False, None, True, B2)

    def _residual(self, f, u):
        return f - (self.A @ u.ravel()).reshape(u.shape)

    # ------------------------------------------------------------- Table 3
    def prec_ud(self, f: np.ndarray) -> np.ndarray:
        """SweepingPrecUD(f)."""
        f = f.reshape(self.nt, self.N)
        u = np.zeros_like(f, dtype=np.complex128)
        B = [None, None]
        self.forward_sweep(u, f, 1, self.J, B)
        g = self._residual(f, u)
        self.backward_sweep(u, g, self.J, 1, B)
        return u.reshape(self.shape)

    def prec_x(self, f: np.ndarray) -> np.ndarray:
        """SweepingPrecX(f), j_mid = J/2 + 1 (J even)."""
        assert self.J % 2 == 0, "the X-sweep needs an even number of subdomains"
        f = f.reshape(self.nt, self.N)
        u = np.zeros_like(f, dtype=np.complex128)
        B1, B2 = [None, None], [None, None]
        jm = self.J // 2 + 1
        self.forward_sweep(u, f, 1, jm - 1, B1)
        self.backward_sweep(u, f, self.J, jm + 1, B2)
        self.mid_solve_in(u, f, jm, B1, B2)
        g = self._residual(f, u)
        self.mid_solve_out(u, g, jm, B2, B1)
        self.backward_sweep(u, g, jm - 1, 1, B1)
        self.forward_sweep(u, g, jm + 1, self.J, B2)
        return u.reshape(self.shape)

    def prec_nx(self, f: np.ndarray, n_cell: int) -> np.ndarray:
        """SweepingPrecNX(f) (Table 3): intersecting sweeps inside n_cell groups
        of subdomains ("cells") separated by the boundary subdomains
        j_cell[1..n_cell-1].

        Readings of the printed listing: j_cell[0] = 0 (with j_cell[n_cell] =
        J + 1, so that n_cell = 1 is SweepingPrecX); a first-phase MidSolveOut
        at a cell boundary sends its layers both ways (right into the next
        cell's forward sweep, B_{2m+1}; left into this cell's backward sweep,
        B_{2m}); the second-phase MidSolveIn of a cell boundary takes the data
        of both neighbouring cells, so it follows all cells' sweeps.
        """
        f = f.reshape(self.nt, self.N)
        jc, jm = nx_layout(self.J, n_cell)
        u = np.zeros_like(f, dtype=np.complex128)
        B = [[None, None] for _ in range(2 * n_cell + 2)]      # B[1] .. B[2 n_cell + 1]
        for m in range(1, n_cell):
            self.mid_solve_out(u, f, jc[m], B[2 * m + 1], B[2 * m])
        for m in range(1, n_cell + 1):
            self.forward_sweep(u, f, jc[m - 1] + 1, jm[m] - 1, B[2 * m - 1])
            self.backward_sweep(u, f, jc[m] - 1, jm[m] + 1, B[2 * m])
            self.mid_solve_in(u, f, jm[m], B[2 * m - 1], B[2 * m])
        g = self._residual(f, u)
        for m in range(1, n_cell + 1):
            self.mid_solve_out(u, g, jm[m], B[2 * m], B[2 * m - 1])
            self.backward_sweep(u, g, jm[m] - 1, jc[m - 1] + 1, B[2 * m - 1])
            self.forward_sweep(u, g, jm[m] + 1, jc[m] - 1, B[2 * m])
        for m in range(1, n_cell):
            self.mid_solve_in(u, g, jc[m], B[2 * m], B[2 * m + 1])
        return u.reshape(self.shape)

    def apply(self, f: np.ndarray, sweep: str = "X", n_cell: int = 2) -> np.ndarray:
        if sweep == "NX":
            return self.prec_nx(f, n_cell)
        return self.prec_x(f) if sweep == "X" else self.prec_ud(f)


def nx_layout(J: int, n_cell: int):
    """Cell boundaries j_cell[0..n_cell] (j_cell[0] = 0, j_cell[n_cell] = J + 1,
    the others equally spaced) and cell centres j_mid[1..n_cell] (j_mid[0]
    unused), for SweepingPrecNX; n_cell = 1 gives the X-sweep's j_mid = J/2 + 1
    for even J."""
    assert 1 <= n_cell <= (J + 1) // 2, "every cell needs at least one subdomain"
    jc = [0] + [int(round(m * (J + 1) / n_cell)) for m in range(1, n_cell)] + [J + 1]
    jm = [0] + [(jc[m - 1] + jc[m] + 1) // 2 for m in range(1, n_cell + 1)]
    for m in range(1, n_cell + 1):
        assert jc[m - 1] < jm[m] < jc[m]
    return jc, jm
