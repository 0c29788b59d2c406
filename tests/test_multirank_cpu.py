"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1).

Ranks shard the instances (disjoint seeds), time is the maximum over ranks,
and the job's throughput counts every rank's units.  No GPU is involved.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import argparse

    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    args = argparse.Namespace(workload="batch", batch_count=8, seed=0)
    seed0 = bench.shard_seed0(args, rank)
    ms = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
    args1 = argparse.Namespace(workload="powerlaw", batch_count=8, seed=5)
    out.put((rank, seed0, bench.shard_seed0(args1, rank), ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, b0, s0, ms0), (r1, b1, s1, ms1) = res
    assert ms0 == ms1 == 20.0                      # maximum over ranks
    assert set(range(b0, b0 + 8)).isdisjoint(range(b1, b1 + 8))   # disjoint batches
    assert s0 != s1


def test_job_throughput_counts_all_ranks():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(2, 4096, 5, 1000.0) == pytest.approx(2 * 4096 * 5)
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
