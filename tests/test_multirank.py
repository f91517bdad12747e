"""The multi-rank path of bench.py with gloo on CPU (world size 2): every rank runs its own
replica, the job time is the maximum over ranks and the value counts every rank's points."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 if rank == 0 else 250.0        # rank 1 is the slow one
    value, max_ms = bench.aggregate_over_ranks(local_ms, points_per_rank=1000, steps=10, dist=dist, device="cpu")
    out[rank] = (value, max_ms)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_max_time_and_summed_points():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        value, max_ms = out[r]
        assert max_ms == 250.0
        assert abs(value - 1000 * 10 * 2 / 0.25) < 1e-9
