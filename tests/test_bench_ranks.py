"""The multi-rank host logic of bench.py on CPU (gloo, world size 2).

Under torchrun every rank solves its own replica; the timed step is the slowest rank's
(maximum over ranks) and the whole-job value counts every rank's DOFs.  The reference arm
runs on rank 0 only.
"""
import contextlib
import io
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        ms = bench.max_over_ranks(100.0 + 25.0 * rank, 2, "cpu")   # rank 1 is the slower replica
        e2e_s = bench.max_over_ranks(0.5 - 0.25 * rank, 2, "cpu")   # rank 0 is the slower one here
        q.put((rank, ms, e2e_s, bench.weak_scaling_value(1000, 2, ms)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_value_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        out = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    for rank, ms, e2e_s, value in out:
        assert ms == 125.0          # both ranks agree on the slowest rank's time
        assert e2e_s == 0.5
        assert value == pytest.approx(1000 * 2 / 0.125)   # all ranks' DOFs / that time


def test_single_rank_passes_values_through():
    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25
    assert bench.weak_scaling_value(345744, 1, 200.0) == pytest.approx(345744 / 0.2)


def test_reference_arm_runs_on_rank_zero_only():
    class Args:
        steps, warmup, ref_iterations = 1, 0, 1

    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.run_reference(Args(), 1, 2) is None   # a non-zero rank exits without work
    assert buf.getvalue() == ""
