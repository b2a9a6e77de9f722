"""Assemble the oracle solver for a ``synth.Workload``.

Fine operator: Eq. 40 (h^d-scaled).  Preconditioner: the sweeping
preconditioner of Table 3 on the fine grid, or (two-grid workloads) the
TGSP of Section 4 with the coarse operator of Appendix A and the sweeping
preconditioner on the coarse grid.  PML constants (reading of Section 2.1):
c_pml = mean wave speed over all unknowns, outer d_pml = w_out h, DD
d_pml = w_dd h_I.
"""

from __future__ import annotations

import numpy as np

from . import dd, fd, fe, gmres, mesh, twogrid


class Problem:
    def __init__(self, cfg, m: np.ndarray | None = None, *, sweep: str | None = None,
                 J: int | None = None, w_dd: int | None = None, s_dd: float | None = None,
                 two_grid: bool | None = None, nu: int | None = None,
                 omega_jac: float | None = None, c_pml: float | None = None,
                 n_cell: int = 2):
        import synth
        self.cfg = cfg
        self.m = synth.medium(cfg) if m is None else np.asarray(m, dtype=np.float64)
        self.sweep = cfg.sweep if sweep is None else sweep
        self.n_cell = n_cell              # cells of the NX-sweep (sweep = "NX")
        self.J = cfg.J if J is None else J
        self.w_dd = cfg.w_dd if w_dd is None else w_dd
        self.s_dd = cfg.s_dd if s_dd is None else s_dd
        self.two_grid = cfg.two_grid if two_grid is None else two_grid
        self.nu = cfg.nu if nu is None else nu
        self.omega_jac = cfg.omega_jac if omega_jac is None else omega_jac
        self.omega = cfg.omega
        h = cfg.h
        # "typical velocity" of the PML (Section 2.1): mean wave speed unless fixed
        self.c_pml = float(np.mean(1.0 / np.sqrt(self.m))) if c_pml is None else float(c_pml)
        # outer boundary layers: PML (Eq. 5), or a sponge (Section 2.1: k ->
        # k (1 + i beta), no PML: alpha = 1) with the standard two-grid cycle of
        # Section 4.1 (every cell coarsened)
        self.boundary = getattr(cfg, "boundary", "pml")
        sponge = self.boundary == "sponge"
        s_out = 0.0 if sponge else cfg.s_out
        self.axes = [mesh.fine_axis(c + 2 * cfg.w_out, cfg.w_out, h, s_out, self.c_pml)
                     for c in cfg.cells]
        self.sponge = np.ones(cfg.shape)
        if sponge:
            bmax = mesh.sponge_beta_max(cfg.sponge_damping, self.omega / self.c_pml, cfg.w_out * h)
            self.sponge = mesh.sponge_factor([mesh.sponge_beta(c + 2 * cfg.w_out, cfg.w_out, h, bmax)
                                              for c in cfg.cells])
        self.k2 = self.omega ** 2 * self.m * self.sponge
        self.A = fd.assemble(self.axes, self.k2, self.omega)
        if self.two_grid:
            if sponge:     # standard coarsening: all cells merged in pairs, no PML
                co = [mesh.coarse_axis(c + 2 * cfg.w_out, 0, h, 0.0, self.c_pml)
                      for c in cfg.cells]
            else:
                co = [mesh.coarse_axis(c, cfg.w_out, h, cfg.s_out, self.c_pml) for c in cfg.cells]
            self.caxes = [c[0] for c in co]
            self.k2c = fe.coarse_k2(self.k2, [c[1] for c in co], [c[2] for c in co])
            H = 2.0 * h
            omega = self.omega

            def builder(axes, med):
                return fe.assemble(axes, med, omega, H)

            self.Ac = builder(self.caxes, self.k2c)
            self.P = fe.prolongation([fe.prolongation_1d(c[1], c[2], N)
                                      for c, N in zip(co, cfg.shape)])
            self.dd = dd.SweepingDD(self.caxes, self.k2c, "cell", builder, self.Ac, self.J,
                                    self.w_dd, self.s_dd, self.c_pml, omega)
        else:
            omega = self.omega

            def builder(axes, med):
                return fd.assemble(axes, med, omega)

            self.dd = dd.SweepingDD(self.axes, self.k2, "node", builder, self.A, self.J,
                                    self.w_dd, self.s_dd, self.c_pml, omega)

    def precondition(self, r: np.ndarray) -> np.ndarray:
        r = np.asarray(r).ravel()
        if self.two_grid:
            out = twogrid.tgsp(r, self.A, self.P, lambda rc: self.dd.apply(rc, self.sweep, self.n_cell),
                               self.nu, self.omega_jac)
        else:
            out = self.dd.apply(r, self.sweep, self.n_cell)
        return np.asarray(out).ravel()

    def apply(self, u: np.ndarray) -> np.ndarray:
        return self.A @ np.asarray(u).ravel()

    def solve(self, b: np.ndarray, m: int | None = None, tol: float | None = None,
              max_iter: int = 500):
        """GMRES(m) to relative residual ``tol``; returns (u, info) per right-hand side."""
        m = self.cfg.gmres_m if m is None else m
        tol = self.cfg.tol if tol is None else tol
        b = np.asarray(b)
        single = b.ndim == self.cfg.dim
        bs = b[None] if single else b
        us, infos = [], []
        for rhs in bs:
            u, info = gmres.gmres(self.apply, rhs.ravel(), self.precondition, m=m, tol=tol,
                                  max_iter=max_iter)
            us.append(u.reshape(self.cfg.shape))
            infos.append(info)
        return (us[0], infos[0]) if single else (np.stack(us), infos)
