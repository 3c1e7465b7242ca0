"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas, no data-path collective).

Each rank reports its own timed milliseconds.  The job value must use the
slowest rank (max over ranks) and count the steps of every rank.
"""

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = [400.0, 500.0][rank]  # rank 1 is the slow replica
    value, total = bench.aggregate_over_ranks(local_ms, steps=20, world=world, dist=dist)
    out[rank] = (value, total)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_uses_slowest_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    for rank in range(world):
        value, total = out[rank]
        assert total == 500.0
        assert value == pytest.approx(2 * 20 / 0.5)


def test_single_rank_is_local_time():
    import bench

    value, total = bench.aggregate_over_ranks(250.0, steps=10, world=1)
    assert total == 250.0 and value == pytest.approx(40.0)
