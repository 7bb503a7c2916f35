"""The benchmark's multi-rank logic on CPU with two gloo ranks (world size 2).

On GPUs every rank of ``bench.py`` is an independent replica (designs shard with
no data-path exchange); the only collectives are the barrier and the maximum of
the timed milliseconds.  Here two CPU processes run that aggregation and the
reference arm's rank rule, over gloo on 127.0.0.1.
"""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 150.0][rank]  # rank 1 is the slower replica
    m = bench.max_over_ranks(ms, world)
    value = bench.job_mlups(world, 1.0e6, 4, m)
    dist.destroy_process_group()
    out.put((rank, m, value))


def test_max_over_ranks_and_job_throughput():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, value in res:
        assert m == 150.0  # every rank sees the slowest rank's time
        # 2 replicas x 1e6 updates x 4 steps over 0.15 s
        assert value == pytest.approx(2 * 1.0e6 * 4 / 0.150 / 1e6)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, 1) == 42.0
    assert bench.job_mlups(1, 2.0e6, 3, 1000.0) == pytest.approx(6.0)


def _reference_rank(rank, out):
    sys.path.insert(0, ROOT)
    os.environ["RANK"] = str(rank)
    import argparse

    import bench
    import io
    import contextlib
    buf = io.StringIO()
    args = argparse.Namespace(gpus=2, steps=1, warmup=0, workload="config1")
    with contextlib.redirect_stdout(buf):
        if rank != 0:
            bench.run_reference(args)
    out.put((rank, buf.getvalue()))


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun the reference arm runs on rank 0 alone; other ranks return
    at once and print nothing."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_reference_rank, args=(1, q))
    p.start()
    rank, text = q.get(timeout=120)
    p.join(timeout=60)
    assert p.exitcode == 0 and rank == 1 and text == ""
