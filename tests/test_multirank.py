"""Host logic of the multi-rank benchmark (replicas only) as world-size-2 gloo ranks on CPU."""
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_local = 1.0 + rank          # rank 1 is the slow one
    dist.barrier()
    t = bench.max_over_ranks(t_local, world, "cpu")
    q.put((rank, t, bench.job_rate(1000, 10, world, t)))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29613
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, rate in res:
        assert t == 2.0                       # max over ranks, on every rank
        assert rate == pytest.approx(1000 * 10 * 2 / 2.0 / 1e6)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
