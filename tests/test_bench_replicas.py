"""The benchmark's N > 1 host logic on CPU.  The path does not shard: N ranks are N
replicas, each rendering its own frame stream of the same data with no data-path
collective.  Gloo ranks with different frame times and ray counts: the whole-job rate is
all ranks' rays over the slowest rank's time."""
import os
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_max, value = bench.replica_rate(1000.0 + 500.0 * rank, 2_000_000 * (rank + 1), dist, "cpu")
        out[rank] = (t_max, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replica_rate_over_gloo(world):
    port = 29517 + world
    out = mp.get_context("spawn").Manager().dict()  # no fork of this multi-threaded process
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    t_slowest = 1000.0 + 500.0 * (world - 1)
    rays = sum(2_000_000 * (r + 1) for r in range(world))
    for r in range(world):
        t_max, value = out[r]
        assert t_max == t_slowest
        assert abs(value - rays / (t_slowest / 1e3) / 1e6) < 1e-9


def test_replica_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.replica_rate(250.0, 1_000_000) == (250.0, 4.0)
