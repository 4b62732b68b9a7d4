"""The N-GPU bench path on the CPU: two gloo ranks stand in for two GPUs.

bench.py runs N independent replicas of the one-GPU step (the path needs no data
exchange), times each with CUDA events, and reports the units all ranks processed
over the slowest rank's time.  Here each rank reports a different fake time: every
rank must see the maximum, the whole-job rate must count both ranks' units over it,
and the reference arm must print nothing on rank 1.
"""
import contextlib
import io
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        ms_local = 100.0 + 25.0 * rank
        ms = bench.max_over_ranks(ms_local, ws, "cpu")
        rate = bench.job_rate(1000.0, ws, ms)
        out = io.StringIO()
        if rank == 1:   # the reference arm runs on rank 0 only; rank 1 must return at once
            with contextlib.redirect_stdout(out):
                bench.reference_arm(None, ws, rank)
        q.put((rank, ms, rate, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_time_and_the_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, rate0, _), (r1, ms1, rate1, out1) = res
    assert ms0 == ms1 == 125.0
    assert rate0 == rate1 == pytest.approx(2 * 1000.0 / 0.125)
    assert out1 == ""


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, 1, "cpu") == 42.0
    assert bench.job_rate(500.0, 1, 250.0) == pytest.approx(2000.0)
