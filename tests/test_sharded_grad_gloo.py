"""Sources of one gradient split over ranks (paper_1412_0464_gb300/distributed.py),
on the CPU with gloo: the shares tile the sources, and the summed misfit and
gradient of 2 and 3 ranks (uneven shares, one rank without sources) equal the
one-rank result.  The per-rank gradient here is the oracle's (exact solves), so
that the exchange logic is tested without a GPU."""

import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_shares_tile_the_sources():
    from paper_1412_0464_gb300.distributed import shard
    for n in (0, 1, 7, 8, 9):
        for world in (1, 2, 3, 5):
            parts = [shard(n, r, world) for r in range(world)]
            assert [i for p in parts for i in p] == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem():
    import synth
    from oracle import adjoint, problem
    cfg = synth.adjoint_workload_2d(32)
    m_true, m0 = synth.medium(cfg, "true"), synth.medium(cfg, "start")
    c_pml = float(np.mean(1.0 / np.sqrt(m0)))
    src = np.array([int(i) * cfg.N + int(j) for i, j in synth.source_nodes(cfg)])
    rec = synth.receivers(cfg)
    d = adjoint.synthetic_data(problem.Problem(cfg, m_true, two_grid=False, c_pml=c_pml), src, rec)
    p0 = problem.Problem(cfg, m0, two_grid=False, c_pml=c_pml)

    def grad_fn(s, r, dd):
        phi, g, _ = adjoint.misfit_and_gradient(p0, s, r, dd)
        return phi, g

    return cfg, src, rec, d, grad_fn


def _worker(rank, ws, port, n_src, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from paper_1412_0464_gb300.distributed import sharded_grad
    cfg, src, rec, d, grad_fn = _problem()
    src, d = src[:n_src], d[:n_src]
    phi, g = sharded_grad(grad_fn, src, rec, d, cfg.shape)
    out[rank] = (phi, g.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("ws,n_src", [(2, 8), (3, 8), (3, 2)])
def test_sharded_gradient_equals_one_rank(ws, n_src):
    sys.path.insert(0, ROOT)
    cfg, src, rec, d, grad_fn = _problem()
    phi1, g1 = grad_fn(src[:n_src], rec, d[:n_src])
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_worker, args=(ws, port, n_src, out), nprocs=ws, join=True,
                       start_method="spawn")
    for r in range(ws):
        phi, g = out[r]
        assert abs(phi - phi1) <= 1e-12 * phi1
        assert np.abs(g - g1).max() <= 1e-12 * np.abs(g1).max()
