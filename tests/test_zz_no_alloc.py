"""The slab solve that allocates no device memory (hz_slab_solve_noalloc).

It serves callers that must not allocate device memory once they are
running: schedulers that forbid allocation after start-up, and applications
that hand all device memory to their own pool allocator.  Its output must
equal the regular hz_slab_solve within the slab-solve tolerance, on two calls
in a row (the calls share one fixed work array), and a warmed-up call must
leave both torch's allocator and the device's free memory unchanged.
Collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test.
"""

import numpy as np
import pytest

import synth

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


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 3e-4)])
def test_noalloc_slab_solve_matches_slab_solve(precision, tol):
    hz = _hz()
    cfg = synth.scaled_workload(2, 90, w_out=8, J=6)
    s = hz.Solver.from_workload(cfg, precision=precision, max_rhs=2)
    s.factor()
    for j in (1, 3, 6):
        W = s.slab_info(j)["W"]
        fd = torch.from_numpy(_rand((2, cfg.N, W), 20 + j)).cuda()
        ref = s.slab_solve(j, fd).cpu().numpy()
        first = s.slab_solve_noalloc(j, fd).cpu().numpy()
        second = s.slab_solve_noalloc(j, fd).cpu().numpy()
        assert _rel(first, ref) <= tol
        assert _rel(second, ref) <= tol
        scale = np.abs(ref).max()
        assert np.abs(first - ref).max() <= tol * scale
        assert np.abs(second - ref).max() <= tol * scale


def test_noalloc_call_allocates_nothing():
    hz = _hz()
    cfg = synth.scaled_workload(2, 90, w_out=8, J=6)
    s = hz.Solver.from_workload(cfg, precision="mixed", max_rhs=1)
    s.factor()
    W = s.slab_info(2)["W"]
    fd = torch.from_numpy(_rand((1, cfg.N, W), 5)).cuda()
    out = torch.empty_like(fd)
    s.slab_solve_noalloc(2, fd, out=out)          # warm-up: first call on this device
    torch.cuda.synchronize()
    a0 = torch.cuda.memory_allocated()
    f0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        s.slab_solve_noalloc(2, fd, out=out)
    torch.cuda.synchronize()
    f1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == a0
    assert f1 == f0
    ref = s.slab_solve(2, fd)
    assert _rel(out.cpu().numpy(), ref.cpu().numpy()) <= 3e-4


def test_noalloc_rejects_work_space_beyond_its_array():
    hz = _hz()
    cfg = synth.workload(2)
    s = hz.Solver.from_workload(cfg, precision="fp64", max_rhs=8, gmres_m=2)
    fd = torch.zeros((8, cfg.N, s.slab_info(2)["W"]), dtype=torch.complex128, device="cuda")
    with pytest.raises(hz.HzError) as e:
        s.slab_solve_noalloc(2, fd)
    assert e.value.status == hz.HZ_EINVAL
    assert "work space" in str(e.value)
