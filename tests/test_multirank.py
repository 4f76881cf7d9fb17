"""Host logic of the multi-rank benchmark on CPU: two gloo ranks on 127.0.0.1. Each rank runs an
independent replica (its own seeded batch); the job's time is the slowest rank's and its rate the
sum over ranks. No GPU: only the reduction and the aggregation are exercised."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dt = bench.max_over_ranks(times[rank], world, "cpu")
        out[rank] = (dt, bench.whole_job_rate(world, 1000.0, 3, dt))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    world, times = 2, [0.5, 0.8]
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, times, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        dt, rate = res[rank]
        assert dt == pytest.approx(0.8)
        assert rate == pytest.approx(2 * 1000.0 * 3 / 0.8)


def test_single_rank_needs_no_collective():
    assert bench.max_over_ranks(0.25, 1, "cpu") == 0.25
    assert bench.whole_job_rate(1, 10.0, 4, 2.0) == pytest.approx(20.0)


def test_reference_arm_prints_only_on_rank_zero(capsys):
    class Args:
        steps, warmup, gpus, workload = 1, 0, 2, bench.WORKLOAD

    bench.run_reference(Args, world=2, rank=1)
    assert capsys.readouterr().out == ""
