"""The N > 1 benchmark path on the CPU: two gloo ranks (world size 2).

The butterfly of one operator does not shard without an all-to-all at the switch
level, so more GPUs run independent replicas; the only cross-rank steps are the
barrier and the max-over-ranks timing that turn per-rank times into the whole-job
rate.  These tests run those steps with the gloo backend, and check that the
reference arm prints from rank 0 only.
"""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        dist.barrier()
        ms_local = 10.0 * (rank + 1)        # rank 1 is the slower replica
        ms = bench.max_over_ranks(ms_local, dist, "cpu")
        rate = bench.whole_job_rate(1000.0, ms, world)
        # the reference arm: only rank 0 prints its line
        args = type("A", (), {"gpus": world, "steps": 1, "warmup": 0})()
        buf = io.StringIO()
        if rank != 0:
            with redirect_stdout(buf):
                bench.run_reference(args, rank, world)
        q.put((rank, ms, rate, buf.getvalue()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_takes_the_slowest_rank_and_sums_the_work():
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
    for rank, ms, rate, out in res:
        assert ms == pytest.approx(20.0)           # max over ranks, on every rank
        assert rate == pytest.approx(2 * 1000.0 / 0.020)  # both ranks' units / the slowest time
        assert out == ""                          # rank 1 of the reference arm is silent


def test_single_process_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(1e6, 500.0, 1) == pytest.approx(2e6)
