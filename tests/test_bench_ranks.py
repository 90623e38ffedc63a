"""Replica runs under torchrun: the whole-job rate aggregates over ranks
(units summed, slowest rank's time), checked with two gloo ranks on CPU."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rate, ms, units = bench.aggregate_rate(10.0 + rank, 100.0 * (rank + 1), dist, "cpu")
    q.put((rank, rate, ms, units))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, rate, ms, units in res:
        assert ms == 200.0 and units == 21.0
        assert rate == pytest.approx(21.0 / 0.2)


def test_single_rank_aggregation():
    sys.path.insert(0, ROOT)
    import bench
    rate, ms, units = bench.aggregate_rate(5, 250.0)
    assert rate == pytest.approx(20.0) and ms == 250.0
