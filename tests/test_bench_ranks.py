"""The multi-rank glue of bench.py on CPU: two gloo ranks (replicas), the job
time is the slowest rank's and the rate counts every rank's solves."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench._dist_setup(None)
        assert (w, r, local) == (world, rank, rank)
        t = bench.max_over_ranks(1.0 + rank, dist, device="cpu")  # rank 1 is the slower one
        out[rank] = (t, bench.job_rate(w, 10, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_and_count_both():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t, rate = out[r]
        assert t == 2.0
        assert rate == pytest.approx(world * 10 / 2.0)


def test_reference_arm_line():
    """The reference arm (the oracle solving the same workload on the host) at a
    small level prints one JSON line with the contract's keys."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--level", "3", "--steps", "2",
                          "--warmup", "1"], cwd=root, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["steps"] == 2 and d["warmup"] == 1  # every requested step runs
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_roofline_object():
    """The roofline of a form's dominant kernel: algorithmic bytes over the launch's
    mean time against the peak, with the per-launch figures it came from."""
    import bench
    table = {"bf16": {"kernel_ms": {"phase1": 0.040, "phase2": 0.030}, "phase1_gbs": 3700.0, "phase2_gbs": 5000.0,
                      "phase1_bytes": 148e6, "phase2_bytes": 150e6}}
    r = bench._roofline(table, "bf16", 99, 6800.0, "measured")
    assert r["kernel"] == "k_phase1<bf16>" and r["achieved"] == 3700.0
    assert r["frac"] == pytest.approx(3700.0 / 6800.0) and r["launch_us"] == pytest.approx(40.0)
    assert r["traffic"] is None  # no capture for this level
