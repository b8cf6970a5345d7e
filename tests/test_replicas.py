"""Multi-GPU runs are replicas (one propagation per rank, no data-path
collective): the host logic of `bench.py --gpus N` on world-size-2 `gloo`
process groups on the CPU."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) seconds: the job time is the slowest rank's
        t = bench.max_over_ranks(1.0 + rank, dist, "cpu")
        rate = bench.job_rate(1000.0, 3, world, t)
        # each rank draws its own replica of the workload (seed 2 + rank)
        prob = bench.I.workload("C1", L=1e-3, seed=2 + rank)
        q.put((rank, t, rate, float(abs(prob.A0).sum())))
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_rate_counts_every_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, t, rate, _ in out:
        assert t == pytest.approx(2.0)
        assert rate == pytest.approx(1000.0 * 3 * 2 / 2.0)
    assert out[0][3] != out[1][3]  # different replicas


def test_single_process_needs_no_process_group():
    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.job_rate(10.0, 2, 1, 4.0) == pytest.approx(5.0)
