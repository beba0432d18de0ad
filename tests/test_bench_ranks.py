"""The multi-rank host logic of bench.py (replicas only: each rank solves its
own copy of the workload; the job's time is the slowest rank's and its
throughput the sum over ranks), run as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank            # rank 1 is the slow one
        got = bench.max_over_ranks(ms, world, "cpu")
        q.put((rank, got, bench.job_rate(100.0, got, world)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]               # every rank sees the slowest time
    assert out[0][2] == pytest.approx(2 * 100.0 / 15e-3)      # world x per-rank cells / slowest time


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_rate(50.0, 10.0, 1) == pytest.approx(5000.0)
