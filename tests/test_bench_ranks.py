"""bench.py's multi-rank logic on CPU: two gloo ranks (replicas) agree on the
slowest rank's time and on the whole-job rate, and the reference arm prints
from rank 0 only."""
import os
import socket
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, str(ROOT))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, l = bench.rank_info()
        ms = 10.0 + 5.0 * rank                       # rank 1 is the slow one
        worst = bench.max_over_ranks(ms, w, device="cpu")
        rate = bench.whole_job_rate(1000, w, worst / 1e3)
        q.put((r, w, l, worst, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[0] for g in got] == [0, 1] and all(g[1] == 2 for g in got)
    assert all(g[3] == 15.0 for g in got)                 # max over ranks
    assert all(abs(g[4] - 2000 / 0.015) < 1e-6 for g in got)  # all ranks' units / slowest time


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, str(ROOT))
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0


def test_reference_arm_prints_from_rank_zero_only(capsys, monkeypatch):
    sys.path.insert(0, str(ROOT))
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        workload, steps, warmup, ref_pixels = "small", 1, 3, 16
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
