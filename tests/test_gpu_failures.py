"""Every failure status of the C ABI, produced without faulting or hanging the GPU.

* HZ_ENOTCONV: a max_iter cap of 1; u holds the last iterate, stats are filled.
* HZ_EINACCURATE: a NaN in the medium (the GMRES residual norm is not finite).
* HZ_ENOMEM: the host-side allocation hook (HZ_TEST_ALLOC_LIMIT) refuses a
  request, in hz_setup and in the first hz_solve_host; nothing leaks into the
  next calls.
* HZ_ETIMEOUT: the fused factorisation's bounded wait (chain progress) gets a
  zero limit (HZ_TEST_WAIT_LIMIT_NS=0): the waiting worker CTAs give up and
  raise the device flag, the chains (which never wait) finish, the launch ends;
  the same handle then factors and solves correctly.
* The separate-launch factorisation (HZ_TEST_NO_COOP=1, used where cooperative
  launch is unavailable) matches the oracle's slab solves.
"""

import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

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


class _env:
    def __init__(self, **kv):
        self.kv = kv

    def __enter__(self):
        for k, v in self.kv.items():
            os.environ[k] = str(v)

    def __exit__(self, *a):
        for k in self.kv:
            os.environ.pop(k, None)


def test_not_converged_returns_last_iterate_and_stats():
    hz = _hz()
    cfg = synth.scaled_workload(2, 90, w_out=8, J=6)
    s = hz.Solver.from_workload(cfg, precision="mixed", max_iter=1)
    s.factor()
    b = torch.from_numpy(synth.sources(cfg)[0]).cuda()
    with pytest.raises(hz.HzError) as e:
        s.solve(b)
    assert e.value.status == hz.HZ_ENOTCONV
    u, st = s.solve(b, check=False)
    assert st["iters_max"] == 1 and 0 < st["relres_max"] < 1
    assert torch.isfinite(u.abs()).all() and float(u.abs().max()) > 0


def test_nan_medium_is_inaccurate():
    hz = _hz()
    cfg = synth.scaled_workload(2, 60, w_out=6, J=4)
    m = synth.medium(cfg).copy()
    m[cfg.N // 2, cfg.N // 3] = np.nan
    s = hz.Solver.from_workload(cfg, m=m, precision="mixed", c_pml=2.0, gmres_m=5, max_iter=10)
    s.factor()
    b = torch.from_numpy(synth.sources(cfg)[0]).cuda()
    with pytest.raises(hz.HzError) as e:
        s.solve(b)
    assert e.value.status == hz.HZ_EINACCURATE


def test_allocation_failure_is_enomem_and_recoverable():
    hz = _hz()
    cfg = synth.scaled_workload(2, 60, w_out=6, J=4)
    with _env(HZ_TEST_ALLOC_LIMIT=1 << 16):
        with pytest.raises(hz.HzError) as e:
            hz.Solver.from_workload(cfg, precision="mixed")
        assert e.value.status == hz.HZ_ENOMEM
    s = hz.Solver.from_workload(cfg, precision="mixed")
    s.factor()
    b = synth.sources(cfg)[0]
    # the staging buffers of the first host-buffer solve are refused
    with _env(HZ_TEST_ALLOC_LIMIT=cfg.ndof * 16):
        with pytest.raises(hz.HzError) as e:
            s.solve_host(torch.from_numpy(b))
        assert e.value.status == hz.HZ_ENOMEM
    u, st = s.solve_host(torch.from_numpy(b))
    p = Problem(cfg)
    exact = spla.spsolve(p.A.tocsc(), b.ravel()).reshape(cfg.shape)
    assert _rel(u.numpy(), exact) <= 1e-5


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_factor_wait_timeout_then_recovery(precision):
    hz = _hz()
    cfg = synth.scaled_workload(2, 300, w_out=10, J=6)
    s = hz.Solver.from_workload(cfg, precision=precision)
    with _env(HZ_TEST_WAIT_LIMIT_NS=0):
        with pytest.raises(hz.HzError) as e:
            s.factor()
        assert e.value.status == hz.HZ_ETIMEOUT
    b = torch.from_numpy(synth.sources(cfg)[0]).cuda()
    with pytest.raises(hz.HzError) as e:           # the failed factorisation does not count
        s.solve(b)
    assert e.value.status == hz.HZ_ENOTFACTORED
    s.factor()
    u, st = s.solve(b)
    assert st["relres_max"] <= cfg.tol
    p = Problem(cfg)
    exact = spla.spsolve(p.A.tocsc(), synth.sources(cfg)[0].ravel()).reshape(cfg.shape)
    assert _rel(u.cpu().numpy(), exact) <= 1e-5


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 3e-4)])
def test_separate_launch_factorisation_matches_oracle(precision, tol):
    hz = _hz()
    cfg = synth.scaled_workload(2, 90, w_out=8, J=6)
    p = Problem(cfg)
    s = hz.Solver.from_workload(cfg, precision=precision, segments=7)
    with _env(HZ_TEST_NO_COOP=1):
        s.factor()
    for j in range(1, cfg.J + 1):
        sl = p.dd.slabs[j]
        fd = _rand((cfg.N, sl.W), 70 + j)
        ud = s.slab_solve(j, torch.from_numpy(fd).cuda()).cpu().numpy()
        ref = sl.lu.solve(fd.ravel()).reshape(fd.shape)
        assert _rel(ud, ref) <= tol
        assert np.abs(ud - ref).max() <= tol * np.abs(ref).max()
