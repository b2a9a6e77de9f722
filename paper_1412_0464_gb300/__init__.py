"""GB300 (sm_103a) Helmholtz solver: GMRES with the improved sweeping
domain-decomposition preconditioner of Stolk (arXiv 1412.0464).

This module is a thin ctypes binding of the C ABI in ``include/hz.h``: it
marshals torch tensors (device memory) and the current CUDA stream into the
library's entry points.  All computation runs in the CUDA library
``_build/libhz.so``; there is no CPU fallback.  Importing the module does not
load the library; the first call does, and fails loudly if it is missing.
"""

from __future__ import annotations

import ctypes
import os
import re

from .build import LIB, build  # noqa: F401

HZ_OK, HZ_EINVAL, HZ_ENOMEM, HZ_ECUDA, HZ_ENOTFACTORED, HZ_ENOTCONV, HZ_ETIMEOUT, HZ_EINACCURATE = range(8)
HZ_SWEEP_UD, HZ_SWEEP_X, HZ_SWEEP_NX = 0, 1, 2
HZ_PLAIN_FP64, HZ_MIXED = 0, 1
HZ_BOUNDARY_PML, HZ_BOUNDARY_SPONGE = 0, 1

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hz.h")


class hz_params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("w_out", ctypes.c_int),
        ("h", ctypes.c_double),
        ("omega", ctypes.c_double), ("s_pml_out", ctypes.c_double), ("s_pml_dd", ctypes.c_double),
        ("J", ctypes.c_int), ("w_dd", ctypes.c_int), ("sweep", ctypes.c_int),
        ("two_grid", ctypes.c_int), ("nu", ctypes.c_int), ("omega_jac", ctypes.c_double),
        ("precision", ctypes.c_int), ("gmres_m", ctypes.c_int), ("max_iter", ctypes.c_int),
        ("tol", ctypes.c_double), ("max_rhs", ctypes.c_int), ("segments", ctypes.c_int),
        ("c_pml", ctypes.c_double), ("n_cell", ctypes.c_int), ("boundary", ctypes.c_int),
        ("sponge_damping", ctypes.c_double), ("block_3d", ctypes.c_int),
    ]


class hz_stats(ctypes.Structure):
    _fields_ = [
        ("n_rhs", ctypes.c_int), ("iters_max", ctypes.c_int), ("relres_max", ctypes.c_double),
        ("t_setup_s", ctypes.c_double), ("t_factor_s", ctypes.c_double),
        ("t_solve_s", ctypes.c_double), ("precond_applies", ctypes.c_longlong),
        ("kernel_launches", ctypes.c_longlong),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_H = ctypes.c_void_p
_SIGNATURES = {
    "hz_setup": (ctypes.c_int, [ctypes.POINTER(hz_params), _P, ctypes.POINTER(_H)]),
    "hz_set_medium": (ctypes.c_int, [_H, _P]),
    "hz_factor": (ctypes.c_int, [_H, _P]),
    "hz_solve": (ctypes.c_int, [_H, _P, _P, ctypes.c_int, _P, ctypes.POINTER(hz_stats)]),
    "hz_solve_host": (ctypes.c_int, [_H, _P, _P, ctypes.c_int, _P, ctypes.POINTER(hz_stats)]),
    "hz_apply": (ctypes.c_int, [_H, _P, _P, ctypes.c_int, _P]),
    "hz_precond": (ctypes.c_int, [_H, _P, _P, ctypes.c_int, _P]),
    "hz_grad": (ctypes.c_int, [_H, _P, ctypes.c_int, _P, ctypes.c_int, _P, _P,
                                      ctypes.POINTER(ctypes.c_double), _P, ctypes.POINTER(hz_stats)]),
    "hz_slab_info": (ctypes.c_int, [_H, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 5),
    "hz_segment_layout": (ctypes.c_int, [ctypes.c_int] * 3 + [ctypes.POINTER(ctypes.c_int)] * 5
                          + [_P, ctypes.c_int, _P, ctypes.c_int]),
    "hz_slab_solve": (ctypes.c_int, [_H, ctypes.c_int, _P, _P, ctypes.c_int, _P]),
    "hz_slab_solve_noalloc": (ctypes.c_int, [_H, ctypes.c_int, _P, _P, ctypes.c_int, _P]),
    "hz_get_stats": (ctypes.c_int, [_H, ctypes.POINTER(hz_stats)]),
    "hz_enable_timing": (ctypes.c_int, [_H, ctypes.c_int]),
    "hz_kernel_timing": (ctypes.c_int, [_H, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.POINTER(ctypes.c_double)]),
    "hz_alu_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), _P]),
    "hz_last_error": (ctypes.c_char_p, [_H]),
    "hz_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "hz_destroy": (None, [_H]),
}

_lib = None


def segment_layout(ny, segments=0, max_auto=304):
    """Layout of the parallel-in-y slab substitution (hz_segment_layout; host
    only): dict with mid, P, S0, NG, G0 and int arrays seg [P, 4] (first row,
    rows, direction, group) and grp [NG, 4] (first segment, last segment, half,
    index within the half)."""
    import numpy as np
    c = [ctypes.c_int() for _ in range(5)]
    code = lib().hz_segment_layout(int(ny), int(segments), int(max_auto),
                                   *[ctypes.byref(x) for x in c], None, 0, None, 0)
    if code != 0:
        raise HzError(code, "hz_segment_layout failed")
    mid, P, S0, NG, G0 = (x.value for x in c)
    seg = np.zeros((P, 4), dtype=np.int32)
    grp = np.zeros((NG, 4), dtype=np.int32)
    code = lib().hz_segment_layout(int(ny), int(segments), int(max_auto),
                                   *[ctypes.byref(x) for x in c], seg.ctypes.data, P,
                                   grp.ctypes.data, NG)
    if code != 0:
        raise HzError(code, "hz_segment_layout failed")
    return dict(mid=mid, P=P, S0=S0, NG=NG, G0=G0, seg=seg, grp=grp)


def alu_peak(precision="mixed", stream=None):
    """Measured FMA throughput of the current device, TFLOP/s (hz_alu_peak):
    FP32 for "mixed", FP64 for "fp64"."""
    v = ctypes.c_double()
    code = lib().hz_alu_peak(HZ_MIXED if precision == "mixed" else HZ_PLAIN_FP64,
                             ctypes.byref(v), _stream(stream))
    if code != HZ_OK:
        raise HzError(code, lib().hz_last_error(None).decode())
    return v.value


def declared_symbols(header: str = HEADER):
    """Function names declared in include/hz.h."""
    txt = open(header).read()
    return sorted(set(re.findall(r"^\s*(?:[\w\*]+\s+)+\**(hz_\w+)\s*\(", txt, re.M)))


def lib():
    """Load libhz.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build it with `python -m paper_1412_0464_gb300.build`"
                               " (the CUDA path has no fallback)")
        L = ctypes.CDLL(LIB)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class HzError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = lib().hz_status_string(status).decode()
        super().__init__(f"{name}: {msg}")


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """One Helmholtz problem on the device: set-up, factorisation and solves.

    ``m`` is the squared slowness 1/c^2 on the unknowns, array order
    ([z][y][x]; torch float64 tensor on the GPU, or anything
    ``torch.as_tensor`` accepts).  ``n`` is the interior cell count along x
    (the sweep axis); ``dims`` (array order, last entry n) gives every axis
    its own count (rectangles, boxes); ``dim`` is 2 or 3.
    """

    def __init__(self, m, *, n, w_out, omega, J, w_dd, s_dd, s_out=20.0, sweep="X",
                 precision="mixed", gmres_m=30, max_iter=500, tol=1e-6, max_rhs=1,
                 two_grid=False, nu=3, omega_jac=0.8, segments=0, c_pml=0.0, dim=2, dims=None,
                 h=0.0, n_cell=2, boundary="pml", sponge_damping=1e-2, block_3d=0):
        import torch
        dims = tuple(dims) if dims is not None else (n,) * dim
        assert len(dims) == dim and dims[-1] == n
        self.dims = dims
        self.N = n + 2 * w_out - 1
        self.shape = tuple(c + 2 * w_out - 1 for c in dims)
        # transverse unknowns of the level that carries the slabs (the coarse
        # level of the two-grid cycle, else the fine grid; the coarse grid of a
        # sponge merges every cell in pairs)
        sponge = boundary == "sponge"
        self.slab_nt = 1
        for c in dims[:-1]:
            if not two_grid:
                self.slab_nt *= c + 2 * w_out - 1
            elif sponge:
                self.slab_nt *= (c + 2 * w_out) // 2 - 1
            else:
                self.slab_nt *= c // 2 + 2 * w_out - 1
        p = hz_params()
        p.dim, p.w_out, p.omega, p.h = dim, w_out, omega, h
        for l, c in enumerate(reversed(dims)):      # hz_params.n is (x, y, z)
            p.n[l] = c
        p.s_pml_out, p.s_pml_dd, p.J, p.w_dd = s_out, s_dd, J, w_dd
        p.sweep = {"X": HZ_SWEEP_X, "UD": HZ_SWEEP_UD, "NX": HZ_SWEEP_NX}[sweep]
        p.n_cell = n_cell
        p.two_grid, p.nu, p.omega_jac = int(two_grid), nu, omega_jac
        p.precision = HZ_MIXED if precision == "mixed" else HZ_PLAIN_FP64
        p.gmres_m, p.max_iter, p.tol, p.max_rhs, p.segments = gmres_m, max_iter, tol, max_rhs, segments
        p.c_pml = c_pml
        p.boundary = {"pml": HZ_BOUNDARY_PML, "sponge": HZ_BOUNDARY_SPONGE}[boundary]
        p.sponge_damping = sponge_damping
        p.block_3d = block_3d
        self.params = p
        md = torch.as_tensor(m, dtype=torch.float64).to("cuda").contiguous()
        assert md.shape == self.shape
        h = _H()
        st = lib().hz_setup(ctypes.byref(p), _ptr(md), ctypes.byref(h))
        if st != HZ_OK:
            raise HzError(st, lib().hz_last_error(None).decode())
        self.h = h
        self.factored = False

    @classmethod
    def from_workload(cls, cfg, m=None, **over):
        import synth
        m = synth.medium(cfg) if m is None else m
        kw = dict(n=cfg.n, w_out=cfg.w_out, omega=cfg.omega, J=cfg.J, w_dd=cfg.w_dd, s_dd=cfg.s_dd,
                  s_out=cfg.s_out, sweep=cfg.sweep, precision=cfg.precision, gmres_m=cfg.gmres_m,
                  tol=cfg.tol, max_rhs=cfg.n_src, two_grid=cfg.two_grid, nu=cfg.nu,
                  omega_jac=cfg.omega_jac, dim=cfg.dim, dims=cfg.cells,
                  boundary=getattr(cfg, "boundary", "pml"),
                  sponge_damping=getattr(cfg, "sponge_damping", 1e-2))
        kw.update(over)
        return cls(m, **kw)

    def _check(self, st):
        if st != HZ_OK:
            raise HzError(st, lib().hz_last_error(self.h).decode())

    def set_medium(self, m):
        """New squared slowness on the same grid (factors must be rebuilt)."""
        import torch
        md = torch.as_tensor(m, dtype=torch.float64).to("cuda").contiguous()
        assert md.shape == self.shape
        self._check(lib().hz_set_medium(self.h, _ptr(md)))
        self.factored = False

    def factor(self, stream=None):
        self._check(lib().hz_factor(self.h, _stream(stream)))
        self.factored = True

    def _field(self, f, cuda=True):
        """(batch [n_rhs, *shape] contiguous, single) for a grid field f of
        shape ``self.shape`` or [n_rhs, *shape], complex128 (the C calls trust
        n_rhs * n_dof elements)."""
        import torch
        if f.dtype != torch.complex128 or f.is_cuda != cuda:
            raise TypeError(f"fields are complex128 {'CUDA' if cuda else 'host'} tensors")
        single = f.dim() == len(self.shape)
        fb = (f[None] if single else f).contiguous()
        if tuple(fb.shape[1:]) != tuple(self.shape):
            raise ValueError(f"field must be [n_rhs, {self.shape}] or {self.shape}, got {tuple(f.shape)}")
        return fb, single

    def solve(self, f, stream=None, check=True):
        """u with A u = f (f: complex128 CUDA tensor [n_rhs, *shape] or shape)."""
        import torch
        fb, single = self._field(f)
        u = torch.empty_like(fb)
        st = hz_stats()
        code = lib().hz_solve(self.h, _ptr(fb), _ptr(u), fb.shape[0], _stream(stream), ctypes.byref(st))
        if check:
            self._check(code)
        return (u[0] if single else u), st.as_dict()

    def solve_host(self, f_host, stream=None, out=None):
        """Same with host (CPU) tensors; the copies are part of the call.  ``out``
        (complex128 host tensor of f's batch shape, pinned for full copy speed)
        receives the solution; otherwise a pageable tensor is allocated."""
        import torch
        fb, single = self._field(f_host, cuda=False)
        if out is None:
            u = torch.empty_like(fb)
        else:
            u = out.reshape(fb.shape) if out.dim() == fb.dim() - 1 else out
            if u.dtype != torch.complex128 or u.is_cuda or tuple(u.shape) != tuple(fb.shape) \
                    or not u.is_contiguous():
                raise ValueError("out must be a contiguous complex128 host tensor shaped like f")
        st = hz_stats()
        self._check(lib().hz_solve_host(self.h, _ptr(fb), _ptr(u), fb.shape[0], _stream(stream),
                                        ctypes.byref(st)))
        return (u[0] if single else u), st.as_dict()

    def apply(self, u, stream=None):
        import torch
        ub, single = self._field(u)
        y = torch.empty_like(ub)
        self._check(lib().hz_apply(self.h, _ptr(ub), _ptr(y), ub.shape[0], _stream(stream)))
        return y[0] if single else y

    def precond(self, r, stream=None):
        import torch
        rb, single = self._field(r)
        z = torch.empty_like(rb)
        self._check(lib().hz_precond(self.h, _ptr(rb), _ptr(z), rb.shape[0], _stream(stream)))
        return z[0] if single else z

    def grad(self, src, rec, d, stream=None, check=True):
        """(Phi, dPhi/dm, stats) for point sources at flat indices ``src``,
        receivers at flat indices ``rec`` and observed data ``d``
        ([n_src, n_rec] complex128); see hz_grad."""
        import torch
        src = torch.as_tensor(src).to(device="cuda", dtype=torch.int32).contiguous()
        rec = torch.as_tensor(rec).to(device="cuda", dtype=torch.int32).contiguous()
        d = torch.as_tensor(d).to(device="cuda", dtype=torch.complex128).contiguous()
        assert d.shape == (src.numel(), rec.numel())
        grad = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        phi = ctypes.c_double()
        st = hz_stats()
        code = lib().hz_grad(self.h, _ptr(src), src.numel(), _ptr(rec), rec.numel(), _ptr(d),
                                    _ptr(grad), ctypes.byref(phi), _stream(stream), ctypes.byref(st))
        if check:
            self._check(code)
        return phi.value, grad, st.as_dict()

    def slab_info(self, j):
        vals = [ctypes.c_int() for _ in range(5)]
        self._check(lib().hz_slab_info(self.h, j, *[ctypes.byref(v) for v in vals]))
        return dict(zip(("lo", "hi", "wl", "wr", "W"), (v.value for v in vals)))

    def _slab_field(self, j, fd, out=None):
        """Checks a slab field [n_rhs, N_t, W] (or [N_t, W]) before the C call,
        which trusts n_rhs * N_t * W complex128 device elements."""
        import torch
        if not isinstance(fd, torch.Tensor) or fd.dtype != torch.complex128 or not fd.is_cuda:
            raise TypeError("slab fields are complex128 CUDA tensors")
        W = self.slab_info(j)["W"]
        nt = self.slab_nt
        fb = (fd[None] if fd.dim() == 2 else fd).contiguous()
        if fb.dim() != 3 or tuple(fb.shape[1:]) != (nt, W):
            raise ValueError(f"slab {j} field must be [n_rhs, {nt}, {W}], got {tuple(fd.shape)}")
        if out is None:
            out = torch.empty_like(fb)
        elif (out.dtype != torch.complex128 or not out.is_cuda or not out.is_contiguous()
              or tuple(out.shape) != tuple(fb.shape)):
            raise ValueError("out must be a contiguous complex128 CUDA tensor shaped like the input")
        return fb, out

    def slab_solve(self, j, fd, stream=None):
        fb, u = self._slab_field(j, fd)
        self._check(lib().hz_slab_solve(self.h, j, _ptr(fb), _ptr(u), fb.shape[0], _stream(stream)))
        return u[0] if fd.dim() == 2 else u

    def slab_solve_noalloc(self, j, fd, stream=None, out=None):
        """slab_solve through the entry point that allocates no device memory
        (``out``, if given, receives the result: then this call allocates
        nothing either)."""
        fb, u = self._slab_field(j, fd, out)
        self._check(lib().hz_slab_solve_noalloc(self.h, j, _ptr(fb), _ptr(u), fb.shape[0],
                                                _stream(stream)))
        return u[0] if fd.dim() == 2 else u

    def enable_timing(self, on=True):
        self._check(lib().hz_enable_timing(self.h, int(on)))

    def kernel_timing(self, tag):
        """(ms, launches, algorithmic bytes) summed over launches of ``tag``."""
        ms, n, b = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
        self._check(lib().hz_kernel_timing(self.h, tag.encode(), ctypes.byref(ms), ctypes.byref(n),
                                           ctypes.byref(b)))
        return ms.value, n.value, b.value

    def stats(self):
        st = hz_stats()
        self._check(lib().hz_get_stats(self.h, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if getattr(self, "h", None):
            lib().hz_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
