"""The multi-rank host logic of bench.py on CPU with the gloo backend,
world size 2: the step time is the maximum over ranks, the ranks share one
K build (column blocks), so the whole-job time per build is the slowest
rank's step time, and the reference arm does its work on rank 0 alone."""
import importlib.util
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        ms = [3.0, 5.0][rank]
        m = b.max_over_ranks(ms, world, "cpu")
        v = b.job_seconds_per_build(m, world)
        dist.barrier()
        out.put((rank, m, v))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(2))
    for rank, m, v in got:
        assert m == 5.0                       # the slower rank's step time
        assert v == pytest.approx(5.0e-3)     # one shared build per step


def test_single_rank_passthrough():
    b = _bench()
    assert b.max_over_ranks(4.25, 1, "cpu") == 4.25
    assert b.job_seconds_per_build(4.0, 1) == pytest.approx(4.0e-3)


def test_reference_arm_runs_on_rank0_only():
    b = _bench()

    class A:
        lmax = 2
        steps = 1
        warmup = 0
        gpus = 2
        workload = "chain"
        ncarbon = 10

    buf = io.StringIO()
    with redirect_stdout(buf):
        assert b.run_reference(A, 1, 2) is None
    assert buf.getvalue() == ""
