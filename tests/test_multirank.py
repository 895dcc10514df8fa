"""The benchmark's multi-rank host logic on CPU ranks (gloo, world size 2): the job time
is the slowest rank's and the throughput counts every rank's units (replicas, weak
scaling, no data-path collective)."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, lr = bench.dist_env()
    assert (r, w, lr) == (rank, world, rank)
    ms = 100.0 + 50.0 * rank                   # rank 1 is the slower one
    cells = 1000 * (rank + 1)
    ms_max, units, value = bench.aggregate(ms, cells, 4, dist, "cpu")
    out[rank] = (ms_max, units, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregate_gloo():
    port = 29500 + os.getpid() % 1000
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for rank in (0, 1):
        ms_max, units, value = out[rank]
        assert ms_max == 150.0 and units == 3000.0
        assert value == pytest.approx(3000.0 * 4 / 0.150)


def test_single_rank_aggregate_without_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(20.0, 500, 2) == (20.0, 500.0, 500 * 2 / 0.02)
