"""The N > 1 path of bench.py (independent replicas, one per rank): the job
time is the max over ranks and the value counts every rank's work.  Run as
two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = [120.0, 150.0][rank]
    m = bench.reduce_max_ms(ms, ws, "cpu")
    v = bench.job_value(1000, 10, ws, m)
    out[rank] = (m, v)
    dist.destroy_process_group()


def test_two_rank_max_and_job_value():
    ws = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    assert out[0][0] == 150.0 and out[1][0] == 150.0
    assert out[0][1] == pytest.approx(3.0 * 1000 * 10 * 2 / 0.150)
    assert out[0][1] == out[1][1]


def test_reference_arm_other_ranks_do_nothing(capsys):
    import bench

    class A:
        steps, warmup, n = 1, 0, 64
    bench.run_reference(A(), ws=2, rank=1)
    assert capsys.readouterr().out == ""


def test_reference_arm_json_line(capsys):
    """Rank 0 of the reference arm prints one JSON line carrying the keys of
    the bench contract, with the oracle's own rate as value, cpu_baseline and
    e2e (no host-device copies)."""
    import json

    import bench

    class A:
        steps, warmup, n = 1, 0, 1024
    bench.run_reference(A(), ws=1, rank=0)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] and d["config"]["nx"] == 1024
