"""The multi-GPU form of the benchmark is replicas only (the path has no
exchange step): every rank solves its own copy of the workload and the job
time is the maximum over the ranks.  This checks that aggregation on CPU with
two gloo ranks, as bench.py runs it under torchrun with one rank per GPU."""

import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = 1.25 + rank            # rank r "took" 1.25 + r seconds
    got = bench.max_over_ranks(local, world, device="cpu")
    dist.barrier()
    q.put((rank, got))
    dist.destroy_process_group()


def test_replica_time_is_the_maximum_over_ranks():
    world = 2
    port = 29500 + (os.getpid() % 1000)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 2.25, 1: 2.25}


def test_single_rank_passes_the_value_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
