"""bench.py's multi-rank logic on CPU with world_size-2 gloo ranks: the whole-job rate
is the units all ranks processed over the slowest rank's span, and under torchrun only
rank 0 runs the reference arm (the CPU oracle)."""
import argparse
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r timed 1 + r seconds for 100 (r + 1) units
    rate, t_max, units = bench.job_rate(1.0 + rank, 100.0 * (rank + 1), device="cpu")
    q.put((rank, rate, t_max, units))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_over_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, t_max, units in out:
        assert t_max == 2.0 and units == 300.0
        assert rate == 150.0


def test_job_rate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(0.5, 10.0, device="cpu") == (20.0, 0.5, 10.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun every rank but 0 exits at once, without touching the oracle."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(gpus=2, steps=1, warmup=3, impl="reference")
    assert bench.run_reference(args) == 0
