"""Workload descriptions for the five benchmark configurations.

Grid convention (Section 2.2 of the paper, which counts cells and puts
Dirichlet nodes on the outer boundary): along every axis there are ``n``
interior cells of size ``h = 1/n`` plus ``w_out`` outer-PML cells on each
side, i.e. ``n_cells = n + 2*w_out`` cells and ``n_cells - 1`` unknowns.
Node ``p`` (0..n_cells) sits at ``x = p*h``; nodes 0 and n_cells carry the
Dirichlet condition, unknown index ``i = p - 1``.  The interior box is
``[w_out*h, (n_cells - w_out)*h]``.

The angular frequency is ``omega = 2*pi*c_min/(ppw*h)`` (``ppw`` points per
wavelength at the slowest speed).  Fields are stored ``[rhs][z][y][x]``
(x fastest; x is the sweep axis).
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional, Tuple


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    dim: int
    n: int                  # interior cells per axis
    w_out: int              # outer PML cells per side
    ppw: float              # points per wavelength at c_min
    c_min: float
    medium: str             # "const" | "grf_layer" | "layered3d" | "grf3d"
    corr: float             # correlation length of the random field (cells)
    J: int                  # slabs along x (even)
    w_dd: int               # DD PML width (cells)
    s_dd: float             # DD PML strength S_pml
    s_out: float            # outer PML strength S_pml
    sweep: str              # "X" | "UD"
    two_grid: bool
    nu: int                 # smoothing steps (pre and post)
    omega_jac: float
    gmres_m: int
    tol: float
    n_src: int
    precision: str          # "fp64" | "mixed"
    seed: int
    n_rec: int = 0
    dims: Optional[Tuple[int, ...]] = None   # interior cells per axis (array order z, y, x);
                                            # None: n on every axis; dims[-1] must equal n
    boundary: str = "pml"                    # outer layers: "pml" (Eq. 5) | "sponge"
    sponge_damping: float = 1e-2             # sponge: one-way amplitude damping of the layer

    @property
    def cells(self) -> Tuple[int, ...]:
        """Interior cells per axis, array order (z, y, x); x is the sweep axis."""
        if self.dims is None:
            return (self.n,) * self.dim
        assert len(self.dims) == self.dim and self.dims[-1] == self.n
        return tuple(self.dims)

    @property
    def n_cells(self) -> int:
        """Cells along x (interior + both PML layers)."""
        return self.n + 2 * self.w_out

    @property
    def N(self) -> int:
        """Unknowns along x."""
        return self.n_cells - 1

    @property
    def shape(self) -> Tuple[int, ...]:
        return tuple(c + 2 * self.w_out - 1 for c in self.cells)

    @property
    def ndof(self) -> int:
        return math.prod(self.shape)

    @property
    def h(self) -> float:
        return 1.0 / self.n

    @property
    def omega(self) -> float:
        return 2.0 * math.pi * self.c_min / (self.ppw * self.h)

    @property
    def n_coarse(self) -> int:
        """Interior cells of the coarse grid (PML cells are not coarsened)."""
        return self.n // 2


def _cfg(**kw) -> Workload:
    base = dict(ppw=8.0, c_min=1.5, corr=0.0, sweep="X", two_grid=False, nu=3,
                omega_jac=0.8, gmres_m=30, tol=1e-6, n_src=1, precision="mixed",
                s_out=20.0, n_rec=0)
    base.update(kw)
    return Workload(**base)


CONFIGS = {
    # 2-D, constant c = 1, 10 ppw, J = 4, sweeping preconditioner alone, c128.
    1: _cfg(name="c1_2d_const_200+10", dim=2, n=200, w_out=10, ppw=10.0, c_min=1.0,
            medium="const", J=4, w_dd=4, s_dd=20.0, gmres_m=20, precision="fp64",
            seed=1412001),
    # 2-D random field + layer jump, 8 ppw at c_min = 1.5, J = 16.
    2: _cfg(name="c2_2d_grf_1000+20", dim=2, n=1000, w_out=20, medium="grf_layer",
            corr=40.0, J=16, w_dd=4, s_dd=20.0, seed=1412002),
    # 2-D large, two-grid outer iteration, sweeps on the half-resolution grid.
    3: _cfg(name="c3_2d_grf_4000+30_tg", dim=2, n=4000, w_out=30, medium="grf_layer",
            corr=160.0, J=32, w_dd=4, s_dd=20.0, two_grid=True, nu=3, omega_jac=0.8,
            seed=1412003),
    # 3-D layered medium, 32 sources as multiple right-hand sides.
    4: _cfg(name="c4_3d_layered_192+12_32rhs", dim=3, n=192, w_out=12, medium="layered3d",
            corr=8.0, J=12, w_dd=3, s_dd=15.0, n_src=32, seed=1412004),
    # 3-D adjoint gradient with two-grid, 8 sources, 256 receivers.
    5: _cfg(name="c5_3d_grf_256+12_tg_adj", dim=3, n=256, w_out=12, medium="grf3d",
            corr=20.0, J=8, w_dd=3, s_dd=15.0, two_grid=True, nu=3, omega_jac=0.6,
            n_src=8, n_rec=256, seed=1412005),
}


def workload(idx: int) -> Workload:
    return CONFIGS[idx]


def scaled_workload(idx: int, n: int, w_out: Optional[int] = None, J: Optional[int] = None,
                    **over) -> Workload:
    """Same medium recipe and frequency rule at a smaller interior size ``n``."""
    w = CONFIGS[idx]
    kw = dataclasses.asdict(w)
    kw.update(n=n, name=f"{w.name}@n{n}", dims=None)
    if w_out is not None:
        kw["w_out"] = w_out
    if J is not None:
        kw["J"] = J
    if w.corr:
        kw["corr"] = w.corr * n / w.n
    kw.update(over)
    return Workload(**kw)


def adjoint_workload_2d(n: int = 128) -> Workload:
    """2-D analogue of configuration 5 (adjoint gradient): smooth random true
    model in [1.5, 4.5] (correlation 20 cells at n = 256), blurred start model,
    8 sources and 16 receivers on a row two cells into the interior, two-grid
    preconditioner, J = 4."""
    return _cfg(name=f"adj2d_{n}+8", dim=2, n=n, w_out=8, medium="grf3d", corr=20.0 * n / 256,
                J=4, w_dd=4, s_dd=20.0, two_grid=True, nu=3, omega_jac=0.8, n_src=8, n_rec=16,
                gmres_m=30, seed=1412105)
