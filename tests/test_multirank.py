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


def test_reference_arm_line_on_rank0():
    """The oracle arm on rank 0: one JSON line with the median of the timed
    steps, the sample stated, the per-column fit non-negative."""
    import json
    b = _bench()

    class A:
        lmax = 2
        steps = 2
        warmup = 1
        gpus = 1
        workload = "chain"
        ncarbon = 8

    buf = io.StringIO()
    with redirect_stdout(buf):
        b.run_reference(A, 0, 1)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "s" and line["value"] > 0
    assert line["higher_is_better"] is False and line["dtype"] == "f64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and "median of 2 steps" in cb["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_oracle_sample_fit():
    """F + u n extrapolation: the fitted per-column time is non-negative and
    the extrapolated build is at least the sampled work."""
    b = _bench()
    from paper_1708_05353_gb300 import inputs
    s = inputs.alkane(8, lmax=2)
    smp = b.OracleSample(s, 2, pair_stride=4)
    v, th = smp.step()
    assert smp.u >= 0 and smp.F >= 0
    assert v >= th
    assert v >= smp.F + smp.u * s.nocc - 1e-12
