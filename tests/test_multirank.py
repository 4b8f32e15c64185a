"""The multi-rank (torchrun) path of bench.py on the CPU: two gloo ranks.

Every rank samples its own instance (its own seed, no data exchange); the
job's time is the slowest rank's and its value counts every rank's attempts.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slower one
    m = bench.max_over_ranks(local_ms, world)
    v = bench.whole_job_value(world, 1000, 10, m)
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.rank_seed(5489, rank))
    out[rank] = (m, v, tuple(seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_over_the_whole_job():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    for rank in (0, 1):
        m, v, seeds = res[rank]
        assert m == pytest.approx(150.0)  # the slowest rank
        assert v == pytest.approx(2 * 1000 * 10 / 0.150)  # every rank's work over the slowest time
        assert seeds[0] != seeds[1]  # independent instances
    assert res[0] == res[1]


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_value(1, 100, 4, 2.0) == pytest.approx(100 * 4 / 0.002)
