"""bench.py's multi-process aggregation on CPU ranks (gloo, world size 2): the job time is the
slowest rank's, and the value counts every rank's problem (weak scaling, replicas)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    assert bench._dist() == (world, rank, rank)
    step_ms = 10.0 + 5.0 * rank                              # rank 1 is the slow one
    m = bench._max_over_ranks(step_ms, "cpu")
    out[rank] = (m, bench._whole_job_value(world, 64, 10, m))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        m, v = out[r]
        assert m == 15.0
        assert v == pytest.approx(2 * 64 * 64 * 10 / 15e-3 / 1e6)
