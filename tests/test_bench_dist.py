"""The benchmark's multi-rank logic on CPU: two gloo ranks, each timing an
independent replica; the whole-job value counts the units of every rank over
the slowest rank's time."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units = 1000.0 * (rank + 1)
    seconds = 2.0 + rank  # rank 1 is the slowest
    tot, slow = bench.aggregate(units, seconds, world)
    bench.barrier(world)
    out[rank] = (tot, slow, bench.dist_env())
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        tot, slow, env = res[rank]
        assert tot == pytest.approx(3000.0)
        assert slow == pytest.approx(3.0)
        assert env == (rank, rank, world)


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate(5.0, 2.0, 1) == (5.0, 2.0)
