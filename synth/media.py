"""Seeded synthetic media, sources and receivers (NumPy PCG64).

The paper's workloads are the Marmousi model (2-D) and the SEG/EAGE salt
model (3-D); neither dataset is available, so these generators produce
stand-ins with the same kind of structure: smooth random velocity with a
sharp layer jump (2-D), a layered medium with a small random perturbation
and a smooth random medium plus a blurred starting model (3-D).

Every array is returned in the ``[z][y][x]`` layout of ``Workload.shape``.
The medium is returned as the squared slowness ``m = 1/c**2`` on all
unknowns (the outer PML region included).
"""

from __future__ import annotations

import numpy as np

from .configs import Workload

_STREAM_MEDIUM = 1
_STREAM_PERTURB = 2
_STREAM_SOURCES = 3
_STREAM_DIRECTIONS = 4


def _rng(cfg: Workload, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([cfg.seed, stream]))


def _smooth_noise(rng: np.random.Generator, shape, corr: float) -> np.ndarray:
    """White noise convolved (periodically) with exp(-r^2 / (2 corr^2))."""
    w = rng.standard_normal(shape)
    spec = np.fft.rfftn(w)
    freqs = [np.fft.fftfreq(s) for s in shape[:-1]] + [np.fft.rfftfreq(shape[-1])]
    k2 = np.zeros(spec.shape)
    for ax, f in enumerate(freqs):
        sh = [1] * len(shape)
        sh[ax] = f.size
        k2 = k2 + (2.0 * np.pi * f.reshape(sh)) ** 2
    return np.fft.irfftn(spec * np.exp(-0.5 * corr * corr * k2), s=shape, axes=range(len(shape)))


def _blur(field: np.ndarray, sigma: float) -> np.ndarray:
    spec = np.fft.rfftn(field)
    shape = field.shape
    freqs = [np.fft.fftfreq(s) for s in shape[:-1]] + [np.fft.rfftfreq(shape[-1])]
    k2 = np.zeros(spec.shape)
    for ax, f in enumerate(freqs):
        sh = [1] * len(shape)
        sh[ax] = f.size
        k2 = k2 + (2.0 * np.pi * f.reshape(sh)) ** 2
    return np.fft.irfftn(spec * np.exp(-0.5 * sigma * sigma * k2), s=shape, axes=range(len(shape)))


def _unit_interval(g: np.ndarray) -> np.ndarray:
    return (g - g.min()) / (g.max() - g.min())


def velocity(cfg: Workload, which: str = "true") -> np.ndarray:
    shape = cfg.shape
    if cfg.medium == "const":
        return np.full(shape, cfg.c_min)
    if cfg.medium == "grf_layer":
        g = _unit_interval(_smooth_noise(_rng(cfg, _STREAM_MEDIUM), shape, cfg.corr))
        # horizontal layer jump: unknown rows at or below node w_out + 0.6 n
        # (the layer is horizontal: across the first array axis, y in 2-D, z in 3-D)
        y = np.arange(shape[0]).reshape((-1,) + (1,) * (cfg.dim - 1))
        y_layer = cfg.w_out + int(round(0.6 * cfg.cells[0])) - 1
        step = (y >= y_layer).astype(np.float64)
        c = 1.5 + 3.0 * (0.7 * g + 0.3 * step)
        return np.broadcast_to(c, shape).copy()
    if cfg.medium == "layered3d":
        z = np.arange(shape[0]) - (cfg.w_out - 1)
        layer = np.clip((6 * z) // cfg.cells[0], 0, 5)
        c0 = (1.5 + 0.5 * layer).reshape(-1, 1, 1)
        xi = _smooth_noise(_rng(cfg, _STREAM_PERTURB), shape, cfg.corr)
        xi = xi / np.abs(xi).max()
        return np.clip(c0 * (1.0 + 0.05 * xi), 1.5, 4.0)
    if cfg.medium == "grf3d":
        c = 1.5 + 3.0 * _unit_interval(_smooth_noise(_rng(cfg, _STREAM_MEDIUM), shape, cfg.corr))
        if which == "start":
            c = _blur(c, 8.0 * cfg.n / 256.0)
        return c
    raise ValueError(cfg.medium)


def medium(cfg: Workload, which: str = "true") -> np.ndarray:
    """Squared slowness m = 1/c^2 (float64, shape ``cfg.shape``)."""
    c = velocity(cfg, which)
    return np.ascontiguousarray(1.0 / (c * c))


def source_nodes(cfg: Workload) -> np.ndarray:
    """Unknown indices (``n_src`` x dim, axis order z,y,x) of the point sources."""
    n, w = cfg.n, cfg.w_out
    cells = cfg.cells
    if cfg.medium == "const" and cfg.n_src == 1:
        return np.array([[c // 2 + w - 1 for c in cells]])
    rng = _rng(cfg, _STREAM_SOURCES)
    if cfg.dim == 2 and cfg.n_rec > 0:
        # sources on the row two cells into the interior, distinct columns
        xs = rng.choice(np.arange(w, w + n - 1), size=cfg.n_src, replace=False)
        return np.stack([np.full(cfg.n_src, w + 2), np.sort(xs)], axis=1)
    if cfg.dim == 2:
        return np.stack([rng.integers(w + c // 4, w + (3 * c) // 4, size=cfg.n_src)
                         for c in cells], axis=1)
    # 3-D: sources on a horizontal plane near the top of the interior
    zplane = w + (4 if cfg.n_rec == 0 else 2)
    ny, nx = cells[1] - 1, cells[2] - 1
    flat = rng.choice(ny * nx, size=cfg.n_src, replace=False)
    out = np.empty((cfg.n_src, 3), dtype=np.int64)
    out[:, 0], out[:, 1], out[:, 2] = zplane, w + flat // nx, w + flat % nx
    assert np.all(out < np.array(cfg.shape))
    return out


def sources(cfg: Workload) -> np.ndarray:
    """Right-hand sides ``b`` (n_src x shape, complex128).

    A unit point source has ``f = h**-d`` at one node; in the h^d-scaled
    system that both solvers use it is ``b = 1`` at that node.
    """
    b = np.zeros((cfg.n_src,) + cfg.shape, dtype=np.complex128)
    for s, idx in enumerate(source_nodes(cfg)):
        b[(s,) + tuple(int(v) for v in idx)] = 1.0
    return b


def receivers(cfg: Workload) -> np.ndarray:
    """Flat unknown indices of the receivers: a square lattice on the source
    plane (3-D) or an evenly spaced line on the source row (2-D)."""
    if cfg.n_rec == 0:
        return np.zeros(0, dtype=np.int64)
    shape = cfg.shape
    if cfg.dim == 2:
        # a line of receivers on the source row, evenly spaced across the interior
        pos = cfg.w_out - 1 + np.round((np.arange(cfg.n_rec) + 0.5) * cfg.n / cfg.n_rec).astype(np.int64)
        return (cfg.w_out + 2) * shape[1] + pos
    side = int(round(cfg.n_rec ** 0.5))
    assert side * side == cfg.n_rec
    zplane = cfg.w_out + 2
    py = cfg.w_out - 1 + np.round((np.arange(side) + 0.5) * cfg.cells[1] / side).astype(np.int64)
    px = cfg.w_out - 1 + np.round((np.arange(side) + 0.5) * cfg.cells[2] / side).astype(np.int64)
    return ((zplane * shape[1] + py[:, None]) * shape[2] + px[None, :]).reshape(-1)


def fd_directions(cfg: Workload, count: int = 4) -> np.ndarray:
    """Seeded smooth perturbation directions of the squared slowness, unit max."""
    rng = _rng(cfg, _STREAM_DIRECTIONS)
    out = np.empty((count,) + cfg.shape)
    for i in range(count):
        d = _smooth_noise(rng, cfg.shape, max(cfg.corr, 1.0))
        out[i] = d / np.abs(d).max()
    return out
