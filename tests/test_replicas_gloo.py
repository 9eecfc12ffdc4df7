"""The multi-GPU form is replicas only (one independent solve stream per GPU, no
collective on the data path).  bench.py's only collective is the max-over-ranks of
the timed region; checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, dist, "cpu")     # rank 1 is the slower one
    out[rank] = (ms, bench.replica_throughput(10, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, value = out[r]
        assert ms == 150.0                               # every rank sees the slowest time
        assert value == pytest.approx(2 * 10 / 0.150)    # units of both ranks / slowest time


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(42.0, None, "cpu") == 42.0
    assert bench.replica_throughput(5, 1, 500.0) == pytest.approx(10.0)
