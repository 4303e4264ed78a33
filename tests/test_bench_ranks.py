"""Host logic of bench.py's multi-process runs, on CPU with the gloo backend (world size 2).

With N GPUs bench.py runs N independent replicas of the workload (the solver has no
exchange step between GPUs): every rank times its own replica, the timed region is the
slowest rank's (a MAX all-reduce), and the whole-job value is all ranks' units over that
time.  The reference arm runs on rank 0 only; the other ranks print nothing.
"""
import argparse
import os
import socket

import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        m = bench.allmax(ms, dist, "cpu")
        q.put((rank, m, bench.replica_throughput(1000, m, world)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, m, v in out:
        assert m == 15.0
        assert v == pytest.approx(2 * 1000 / 0.015)


def test_single_process_aggregation_is_the_identity():
    assert bench.allmax(3.5) == 3.5
    assert bench.replica_throughput(100, 50.0, 1) == pytest.approx(2000.0)


def test_reference_arm_prints_on_rank_zero_only(capsys):
    args = argparse.Namespace(steps=1, warmup=0)
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""
