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


def test_reference_arm_line_keeps_the_contract():
    """`bench.py --impl reference` on rank 0 (the FP64 oracle on the host cores, a bounded
    sample): one JSON line with the arm's metric, unit and direction, its cpu_baseline
    (kind, cores, sample, value = the line's) and an e2e object with no host-device bytes."""
    import json
    import subprocess
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "acc+gradient interactions/s"
    assert d["unit"] == "interactions/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1 and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
