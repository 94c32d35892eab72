"""The multi-rank pieces of bench.py on CPU.  Two gloo ranks stand in for two
GPUs that run independent replicas (the path does not shard): the job time is
the slowest rank's, the value divides it by the steps of all ranks, every
rank draws its own replica, and the reference arm runs on rank 0 only."""
import argparse
import os
import socket

import pytest

import bench

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sec = bench.max_over_ranks(1.0 + 0.5 * rank, world, "cpu")
        dist.barrier()
        q.put((rank, sec, bench.replica_seed(10, rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=180) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    assert [r[1] for r in res] == [1.5, 1.5]          # max over ranks on every rank
    assert res[0][2] != res[1][2]                      # independent replicas
    assert bench.job_seconds_per_step(1.5, 2, 3) == 0.25


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(0.7, 1, "cpu") == 0.7
    assert bench.job_seconds_per_step(0.7, 1, 7) == pytest.approx(0.1)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.main_reference(argparse.Namespace(workload=bench.DEFAULT_WORKLOAD, steps=1, warmup=0))
    assert capsys.readouterr().out == ""
