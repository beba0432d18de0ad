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


def test_cost_model_with_coarse_composition():
    """Sec. 3.4's T(k) = c k t_num + (2s - k)(k + 1)/2 m t_nn with the unit costs
    taken from the measured phases: m = 1 reproduces the plain model; composing
    G m times multiplies the coarse term by m."""
    s, c, k = 16, 400, 16
    seq_ms = 57.6
    t_nn = 0.44
    calls1 = (2 * s - k) * (k + 1) // 2
    st = {"coarse_calls": calls1, "coarse_ms": calls1 * t_nn}
    one = bench.cost_model(st, seq_ms, [k], 1, s, c, 1)
    t_num = seq_ms / (s * c)
    assert abs(one["T_k_ms"] - (c * k * t_num + calls1 * t_nn)) < 1e-9
    st2 = {"coarse_calls": 2 * calls1, "coarse_ms": 2 * calls1 * t_nn}
    two = bench.cost_model(st2, seq_ms, [k], 1, s, c, 2)
    assert abs(two["t_nn_ms"] - t_nn) < 1e-12
    assert abs(two["T_k_ms"] - (c * k * t_num + 2 * calls1 * t_nn)) < 1e-9
    assert two["S_k"] < one["S_k"]
