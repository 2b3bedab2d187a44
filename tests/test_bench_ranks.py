"""Multi-rank host logic of bench.py on CPU: world_size 2 over gloo.

The path shards as independent replicas, so the only cross-rank step is the
timing reduction (max over ranks) and the whole-job figure derived from it.
"""
import io
import contextlib
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [1.0 + 2.0 * rank, 10.0 - rank]          # rank 0: [1, 10]; rank 1: [3, 9]
        out[rank] = bench.max_over_ranks(mine, world, "cpu") + [bench.job_value(4.0, world)]
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_world2():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    assert out[0] == out[1] == [3.0, 10.0, 2.0]


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks([1.5, 2.5], 1, "cpu") == [1.5, 2.5]
    assert bench.job_value(4.0, 1) == 4.0


def test_reference_arm_silent_on_other_ranks(monkeypatch):
    """Under torchrun only rank 0 runs the oracle arm; the others exit without work."""
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()

    class Args:
        steps, warmup = 1, 3

    with contextlib.redirect_stdout(buf):
        bench.run_reference(Args())
    assert buf.getvalue() == ""
