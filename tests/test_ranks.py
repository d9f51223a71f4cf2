"""The replicas path of the benchmark on two CPU ranks (gloo over
127.0.0.1): the barrier bracketing the timed region, the slowest rank's time
reaching every rank, and the whole-job rate of N replicas."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.sync_ranks(world)  # no device: the barrier alone
        # rank r took 1 + r seconds; every rank must see the slowest
        out[rank] = bench.max_over_ranks(1.0 + rank, world, "cpu")
        bench.sync_ranks(world)
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_job_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        assert dict(out) == {0: 2.0, 1: 2.0}
    # 2 replicas, each 100 units per step for 10 steps, in 2 s: 1000 units/s
    assert bench.job_rate(100, 10, 2, 2.0) == 1000.0


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(0.25, 1) == 0.25
    bench.sync_ranks(1)
