"""bench.py's multi-rank arithmetic on CPU with the gloo backend.

The workload has no exchange step: N ranks run N replicas, and the
whole-job rate is every rank's cells over the slowest rank's time.  Two
gloo ranks check that every rank sees the same maximum and rate, and
that only rank 0 prints the reference line.
"""
import io
import os
import socket
import contextlib

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [120.0, 150.0][rank]
        rate, ms_max = bench.replica_rate(ms, 1000, 10, world, dist, "cpu")
        out[rank] = (rate, ms_max)
    finally:
        dist.destroy_process_group()


def test_replica_rate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]
    rate, ms_max = res[0]
    assert ms_max == 150.0
    assert rate == pytest.approx(2 * 1000 * 10 / 0.150)


def test_single_process_rate():
    rate, ms = bench.replica_rate(100.0, 500, 4, 1)
    assert ms == 100.0 and rate == pytest.approx(500 * 4 / 0.1)


def test_reference_arm_only_rank0_prints(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    class A:
        cpu_sample_n, jitter, steps, warmup, gpus = 4, 0.1, 1, 0, 2
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.reference_arm(A) == 0
    assert buf.getvalue() == ""
