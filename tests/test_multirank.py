"""Multi-rank bookkeeping of bench.py on CPU (gloo, world size 2): replicas report the
slowest rank's time and the summed work; the reference arm runs on rank 0 only."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, work = bench.aggregate_ranks(10.0 + rank, 100.0 * (rank + 1), world, "cpu")
    q.put((rank, ms, work))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 11.0, 300.0), (1, 11.0, 300.0)]


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(5.0, 7.0, 1, "cpu") == (5.0, 7.0)


def test_reference_arm_other_ranks_do_nothing(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    ns = type("A", (), {"workload": "plummer_64k", "warmup": 0, "steps": 1, "dt": 2.0 ** -7,
                        "gpus": 2})()
    bench.run_reference(ns)
    assert capsys.readouterr().out == ""
