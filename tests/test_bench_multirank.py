"""The bench's multi-rank timing logic (max over ranks, whole-job rate) on two gloo ranks (CPU)."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    mine = 1.5 + rank  # seconds: rank 1 is the slowest
    dist.barrier()
    t = bench.reduce_max(mine, dist, torch.device("cpu"))
    rate = bench.whole_job_rate(world, 1000, 10, t)
    out[rank] = (t, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        t, rate = out[rank]
        assert t == pytest.approx(2.5)
        assert rate == pytest.approx(world * 1000 * 10 / 2.5)


def test_single_process_identity():
    import bench

    assert bench.reduce_max(3.0, None, torch.device("cpu")) == 3.0
    assert bench.whole_job_rate(1, 10, 2, 4.0) == 5.0
