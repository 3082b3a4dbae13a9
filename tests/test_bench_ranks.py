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
