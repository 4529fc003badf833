"""The multi-process path of bench.py on CPU: world_size-2 gloo ranks (replicas, no data-path collective).

Each rank times its own replica; the job's time is the maximum over ranks and its rate counts every rank's
systems. The reference arm runs on rank 0 only.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        job_ms = bench.max_over_ranks(times[rank], "cpu")
        out.put((rank, job_ms, bench.whole_job_rate(world, 5, job_ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    times = [120.0, 150.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(out.get(timeout=5) for _ in range(2))
    for rank, job_ms, rate in res:
        assert job_ms == 150.0
        assert rate == pytest.approx(2 * 5 / 0.150)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, "cpu") == 42.0
    assert bench.whole_job_rate(1, 4, 2000.0) == pytest.approx(2.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        workload, steps, warmup, cpu_budget_s = "cant16", 1, 0, 1.0
    bench.run_reference(Args())          # returns at once on a non-zero rank
    assert capsys.readouterr().out == ""
