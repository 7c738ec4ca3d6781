"""Multi-rank host logic of bench.py on CPU: two gloo ranks, each with its own
replica's time and work; the job's time is the slowest rank's and its work
the sum over ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_setup()
        assert (w, r, local) == (world, rank, rank)
        dist.barrier()
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist)        # rank 1 is slower
        work = bench.sum_over_ranks(1000 * (rank + 1), dist)       # replicas of different sizes
        out[rank] = (ms, work, work / (ms * 1e-3))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_agree_on_time_and_work():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1]
    ms, work, value = out[0]
    assert ms == 15.0 and work == 3000.0
    assert value == pytest.approx(3000.0 / 0.015)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.0, None) == 3.0
    assert bench.sum_over_ranks(7.0, None) == 7.0
