"""Multi-rank host logic of bench.py, on CPU with the gloo backend (world size 2).

The solve does not shard: N GPUs run N independent replicas of the problem,
with no exchange on the data path.  What crosses ranks is only the timing:
the whole-job value is the units all ranks processed divided by the slowest
rank's time, and the CPU-oracle arm runs on rank 0 alone.
"""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, ms_by_rank, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        value, ms = bench.replica_value(dist, ws, 1000, 3, ms_by_rank[rank])
        ms64 = bench.max_over_ranks(dist, ms_by_rank[rank] * 2.0)
        out.put((rank, value, ms, ms64))
    finally:
        dist.destroy_process_group()


def _run(ws, ms_by_rank):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, ms_by_rank, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(res)


def test_replica_value_uses_slowest_rank_on_every_rank():
    res = _run(2, [100.0, 250.0])
    for rank, value, ms, ms64 in res:
        assert ms == 250.0 and ms64 == 500.0
        # 2 ranks x 1000 nodes x 3 steps in 0.25 s
        assert value == pytest.approx(2 * 1000 * 3 / 0.25, rel=1e-15)


def test_replica_value_single_process_needs_no_group():
    import bench

    value, ms = bench.replica_value(None, 1, 1000, 3, 150.0)
    assert ms == 150.0 and value == pytest.approx(1000 * 3 / 0.15, rel=1e-15)


def test_reference_arm_does_no_work_off_rank_zero(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    def boom(*a, **k):
        raise AssertionError("the oracle ran on rank 1")

    monkeypatch.setattr(bench, "cpu_baseline_subprocess", boom)

    class A:
        workload, steps, warmup, gpus = "disk_4M_m6_n56", 3, 3, 2

    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
