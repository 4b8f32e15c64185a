"""The multi-rank (torchrun) path of bench.py on the CPU: two gloo ranks.

Every rank samples its own instance (its own seed, no data exchange); the
job's time is the slowest rank's and its value counts every rank's attempts.
In batch mode the 4096 instances are sharded over the ranks instead.
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


def _shard_worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    from paper_1004_0024_gb300 import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    descs = W.ragged_instances(4096)
    mine = bench.shard(descs, rank, world)
    work = sum(d["L"] * d["L"] * d["M"] * d["R"] for d in mine)
    total = bench.sum_over_ranks(work, world)
    slowest = bench.max_over_ranks(10.0 + rank, world)
    out[rank] = ([d["index"] for d in mine], work, total, slowest)
    dist.barrier()
    dist.destroy_process_group()


def test_batch_instances_are_sharded_over_gloo_ranks():
    """Batch mode over N ranks: the 4096 instances are split without overlap
    (rank r takes r, r + N, ...), the job's work is the sum over the ranks and
    its time the slowest rank's (no data exchange between ranks)."""
    ctx = mp.get_context("spawn")
    world = 3
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        mp.start_processes(_shard_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    ids = sorted(i for r in range(world) for i in res[r][0])
    assert ids == list(range(4096))
    assert all(i % world == r for r in range(world) for i in res[r][0])
    total = sum(res[r][1] for r in range(world))
    for r in range(world):
        assert res[r][2] == pytest.approx(total)
        assert res[r][3] == pytest.approx(10.0 + world - 1)
