"""Multi-process logic of bench.py on CPU (gloo, world size 2): replicas only,
the job time is the slowest rank's, the value counts every rank's unknowns,
and the reference arm runs on rank 0 alone."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    assert bench._dist()[:2] == (ws, rank)
    ms, value = bench.replica_throughput(10.0 * (rank + 1), 1.0e6, ws, "cpu")
    out[rank] = (ms, value)
    # the reference arm: ranks other than 0 return at once without work
    if rank != 0:
        class A:
            workload = 2
        out[ws + rank] = bench.reference_arm(A())
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_two_ranks():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_worker, args=(ws, port, out), nprocs=ws, join=True, start_method="spawn")
    assert out[0] == out[1]
    ms, value = out[0]
    assert ms == 20.0                              # max over ranks
    assert abs(value - ws * 1.0e6 / 0.020 / 1e6) < 1e-9   # all ranks' unknowns / job time
    assert out[ws + 1] == 0


def test_single_rank_no_collective():
    import bench
    ms, value = bench.replica_throughput(5.0, 2.0e6, 1, "cpu")
    assert ms == 5.0 and abs(value - 400.0) < 1e-12
