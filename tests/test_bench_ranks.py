"""The multi-rank bookkeeping of bench.py on CPU (gloo, two processes): each rank solves its own
problem (replicas), the job time is the slowest rank's, and the whole-job rate counts every rank's
solves.  Also: the reference arm runs on rank 0 only."""

import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world_size, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world_size))
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    import bench

    slowest = bench._max_over_ranks(10.0 + 5.0 * rank, dist, torch.device("cpu"))
    out[rank] = (slowest, bench._job_rate(world_size, 100, slowest / 1e3))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_both():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    # 10 ms and 15 ms: both ranks report the 15 ms rank; the job solved 2 x 100 problems in 15 ms
    assert res[0] == res[1] == (15.0, pytest.approx(2 * 100 / 0.015))


def test_single_process_needs_no_group():
    import bench

    assert bench._max_over_ranks(7.5, None, None) == 7.5
    assert bench._job_rate(1, 10, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import argparse

    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(argparse.Namespace(steps=1, warmup=1, gpus=2)) == 0
    assert capsys.readouterr().out == ""
