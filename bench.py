#!/usr/bin/env python
"""Benchmark of the far-field occ-FMM-K exchange build on GB300.

Workload (default): the protein-sized cluster C202H317O64N55S6-like (644
atoms by random sequential addition at >= 2.0 bohr in a 45-bohr ellipsoid;
heavy atoms 3s2p, H 2s, 3 primitives with log-uniform exponents in [0.1, 50]),
3577 AOs, nocc = 660 Loewdin-orthonormalised random orbitals, octree to ~8
atoms per leaf (depth 3, 12,330 M2L edges), lmax = 2, plain FP64 -- the
largest workload of the method that fits one GPU.  One "step" = one
occk_farfield_K call (steps a-e: C on the device -> K^ff, E^ff).

The same JSON line also carries: every mixed-precision form on the same
workload (time, speed-up over the FP64 GPU form, errors against the FP64 GPU
result and against exact oracle K columns), the learned per-edge rank
selector against fixed rank 10 (FP64 and split-FP16), the 150-carbon chain
(C150H302) in FP32 and FP16X3, the far-field Coulomb matrix, and
occupied-pair screening on localised orbitals of that chain.

Prints ONE JSON line on rank 0.  `value` = seconds per far-field K build for
the whole job (lower is better).  With N GPUs (torchrun) the ranks share one
build: rank g computes the K columns of its occupied block (every pair that
touches the block), the blocks are gathered over NCCL and E is formed from
the gathered K (strong scaling).  `--impl reference` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("far-field K_ri build time (s) & TFLOP/s at stated error vs FP64 oracle, "
          "learned/mixed vs plain")
GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_columns.npz")
MIXED = ["fp32", "tf32", "bf16", "fp16", "bf16x3", "fp16x3"]
# FP64 with steps (a) and (e) from 7-bit integer slices on the tensor core
# (occk_set_fp64_slices): FP64 arithmetic everywhere else, exact slice sums
SLICED = {"fp64s": 7, "fp64s6": 6}
# FP32 with steps (a) and (e) from 4 integer slices (exact sums) on the tensor core
F32SLICED = {"fp32s": 4}


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="protein", choices=["protein", "chain", "chain-loc", "water", "batch"],
                   help="protein: the 644-atom cluster (default); chain: C{ncarbon}H{2n+2}; chain-loc: the chain "
                        "with localised orbitals, every build screened at --screen-tau")
    p.add_argument("--ncarbon", type=int, default=150)
    p.add_argument("--lmax", type=int, default=2)
    p.add_argument("--prec", default="fp64", help="precision of the headline line")
    p.add_argument("--fp64-slices", type=int, default=0, choices=[0, 6, 7],
                   help="with --prec fp64: steps (a), (e) from this many integer slices on the tensor core and "
                        "the half transform and tree passes in double-FP32 (0: the DFMA form)")
    p.add_argument("--variants", default=",".join(["fp64s", "fp32s"] + MIXED),
                   help="other precisions timed on the same workload (comma list, or 'none')")
    p.add_argument("--learned-rank", type=int, default=10,
                   help="reference rank of the learned-selector comparison on the protein workload (0: skip)")
    p.add_argument("--learned-tau", type=float, default=1e-6, help="error budget (Eh) of the learned selector")
    p.add_argument("--no-chain", action="store_true", help="skip the C150H302 FP32/FP16X3 object")
    p.add_argument("--no-batch", action="store_true", help="skip the uneven-batch object")
    p.add_argument("--screen-tau", type=float, default=1e-4,
                   help="occupied-pair screening threshold timed on localised orbitals of C150H302 (0: skip)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--batch-fp64", action="store_true", help="run the batch workload in FP64 (default FP32)")
    p.add_argument("--tune-cache", default=os.path.join(tempfile.gettempdir(), "occk_batch_tune_cache.txt"),
                   help="autotune cache file of the batch workload (outside the repository by default)")
    return p.parse_args(argv)


def make_system(workload, lmax, ncarbon=150):
    from paper_1708_05353_gb300 import inputs
    if workload == "protein":
        return inputs.protein_like(lmax=lmax)
    if workload == "water":
        return inputs.water(100, lmax=lmax)
    if workload == "chain-loc":
        return inputs.alkane_localised(ncarbon, lmax=lmax)
    return inputs.alkane(ncarbon, lmax=lmax)


GOLDEN_KEY = {("protein", 2): "protein", ("chain", 2): "chain150", ("chain-loc", 2): "chain150loc"}


def golden_columns(workload, L, system):
    """Exact oracle K columns stored for this workload (written by
    tests/golden/make_columns.py from the oracle alone), or None."""
    import numpy as np
    key = GOLDEN_KEY.get((workload, L))
    if key is None or not os.path.exists(GOLDEN):
        return None
    g = np.load(GOLDEN)
    if f"{key}/L{L}/K" not in g:
        return None
    fp = g[f"{key}/fingerprint"]
    cols = g[f"{key}/cols"]
    if int(fp[0]) != system.basis.nao or int(fp[1]) != system.nocc or \
            abs(float(np.sum(system.C[:, cols])) - fp[5]) > 1e-10 * max(1.0, abs(fp[5])):
        return None
    return {"cols": cols, "K": g[f"{key}/L{L}/K"], "E_cols": float(g[f"{key}/L{L}/E_cols"]), "key": key}


def oracle_errors(gold, K, C):
    """Errors of a device K against the oracle's exact columns: max|dK| over
    max|K| on those columns, and |dE| of their part of the energy."""
    import numpy as np
    import torch
    if gold is None:
        return {}
    cols = gold["cols"]
    Kc = K[:, torch.as_tensor(cols, device=K.device)].cpu().numpy()
    Ec = -0.5 * float(np.sum(C[:, cols] * Kc))
    return {"oracle_cols": [int(c) for c in cols],
            "rel_dK_vs_oracle": float(np.max(np.abs(Kc - gold["K"])) / np.max(np.abs(gold["K"]))),
            "abs_dE_cols_vs_oracle_Eh": abs(Ec - gold["E_cols"])}


# ---------------------------------------------------------------------------
# algorithmic FLOPs per stage (real form; only the symmetric half of the
# occupied pairs in (a) O^{ij} and in the tree passes b-d)
# ---------------------------------------------------------------------------
def stage_flops(rowoff, nocc, L, nent, nm2m, nl2l, nm2l, m2l_ranks=None):
    nc = (L + 1) ** 2
    tl = sum((2 * l + 1) * (l + 1) ** 2 for l in range(L + 1))
    P = nocc * (nocc + 1) // 2          # the tree passes need only pairs i <= j
    S = [rowoff[k + 1] - rowoff[k] for k in range(len(rowoff) - 1)]
    if m2l_ranks is None:
        m2l = 2.0 * nc * nc * P * nm2l
    else:
        m2l = sum(2.0 * (r + 1) ** 4 * P for r in m2l_ranks)
    return {
        "a_half": 2.0 * nent * nocc * nc,
        "a_full": sum(2.0 * s * nc * nocc * (nocc + 1) / 2 for s in S),
        "b_m2m": 2.0 * tl * P * nm2m,
        "c_m2l": m2l,
        "d_l2l": 2.0 * tl * P * nl2l,
        "e_l2p": sum(2.0 * s * nc * nocc * nocc for s in S),
        "reduce": 0.0,
    }


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.p = None
        self.dev = device_index
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(device_index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            return None
        rows = [r for r in csv.reader(io.StringIO(out)) if len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, n in enumerate(names):
                if "Active" in r[5 + k] and "Not" not in r[5 + k]:
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def max_over_ranks(x, world, device):
    """The largest value of x over the ranks (all_reduce MAX); x itself on
    one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_seconds_per_build(ms_max, world):
    """Whole-job time per far-field K build.  The ranks share one build (each
    computes its column block), so the slowest rank's step time is the time of
    one whole K build, whatever the number of ranks."""
    return ms_max * 1e-3


def function_source(path, name):
    """Text of the C++ function `name` in `path`: from its signature line to the
    first closing brace at column 0."""
    text = open(path).read()
    i = text.index(" " + name + "(")
    i = text.rfind("\n", 0, i) + 1
    j = text.index("\n}\n", i) + 3
    return text[i:j]


def traffic_for(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current source of the kernel's function."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get(kernel)
        if not rec:
            return None
        src = os.path.join(ROOT, "paper_1708_05353_gb300", "csrc", rec["source"])
        body = function_source(src, rec["function"])
        sha = hashlib.sha256(body.encode()).hexdigest()[:16]
        if sha != rec["source_sha"]:
            return None
        return rec["bytes_per_launch"] * rec.get("scale_to_bench", 1.0)
    except Exception:
        return None


def blas_name():
    try:
        import numpy as np
        b = np.show_config(mode="dicts")["Build Dependencies"]["blas"]
        return f"{b.get('name')} {b.get('version')}"
    except Exception:
        return "unknown"


# ---------------------------------------------------------------------------
# The FP64 oracle on a bounded sample of one build (CPU baseline and the
# reference arm).  Like the GPU arm's timed region, a build here is steps
# (a)-(e): the AO->MO half transform and, for every occupied column, the full
# transform, M2M, M2L, L2L and K (the tree and the AO-pair multipoles, step
# a0, are per-geometry set-up on both sides).  The half transform costs the
# same for every shell pair, so it is timed on every `pair_stride`-th pair and
# scaled up; steps 1b-5 for a set of c columns cost F + u c (F: the operators
# the oracle builds per edge and box and its loops over them, u: the work per
# column), with F and u fitted once at 1 and 3 columns.  A step re-times the
# half-transform sample and adds F + u nocc.  The values of a sampled half
# transform are incomplete; only its time is used.
# ---------------------------------------------------------------------------
class OracleSample:
    def __init__(self, system, L, pair_stride=64):
        import numpy as np
        from oracle import fmm
        from oracle import tree as otree
        self.fmm = fmm
        self.system, self.L = system, L
        t0 = time.perf_counter()
        tr = otree.build_tree(system.basis, system.depth, system.target_atoms_per_leaf)
        self.npair = len(tr["pair_a"])
        self.stride = max(1, min(pair_stride, self.npair))
        sub = np.arange(0, self.npair, self.stride)
        self.tr = dict(tr)
        for k in ("pair_a", "pair_b", "leaf_of_pair"):
            self.tr[k] = tr[k][sub]
        self.scale = self.npair / len(sub)
        self.Op = fmm.pair_multipoles(system.basis, self.tr, L)
        self.t_setup = time.perf_counter() - t0
        self.W = None
        self.time_half()
        n3 = max(1, min(3, system.nocc))
        self.t1 = self.time_cols([0])
        self.t3 = self.time_cols(list(range(n3))) if n3 > 1 else self.t1
        self.u = max((self.t3 - self.t1) / (n3 - 1), 0.0) if n3 > 1 else self.t1
        self.F = max(self.t1 - self.u, 0.0)
        self.t_fit = self.t1 + self.t3

    def time_half(self):
        t0 = time.perf_counter()
        self.W = self.fmm.half_transform(self.system.basis, self.tr, self.Op, self.system.C, self.L)
        return time.perf_counter() - t0

    def time_cols(self, cols):
        t0 = time.perf_counter()
        self.fmm.farfield(self.system, L=self.L, tree=self.tr, i_subset=list(cols), Opair=self.Op, W=self.W)
        return time.perf_counter() - t0

    def step(self):
        """One sample: the half transform on the pair sample, timed now;
        returns (extrapolated build seconds, that time)."""
        th = self.time_half()
        return th * self.scale + self.F + self.u * self.system.nocc, th

    def describe(self, th):
        return (f"oracle FP64 on {self.system.name} L={self.L}, steps (a)-(e): half transform timed on 1/"
                f"{self.stride} of the {self.npair} shell pairs ({th:.2f} s, x{self.scale:.1f}) plus steps "
                f"1b-5 for all {self.system.nocc} columns as F + u n with F = {self.F:.2f} s, u = {self.u:.3f} "
                f"s per column, fitted at 1 and 3 columns ({self.t1:.2f} s, {self.t3:.2f} s); set-up "
                f"outside the build (tree, pair multipoles of the sample): {self.t_setup:.1f} s")


def cpu_baseline(system, L, pair_stride=64):
    smp = OracleSample(system, L, pair_stride)
    v, th = smp.step()
    return {"value": v, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": smp.describe(th), "blas": blas_name(),
            "blas_threads": os.environ.get("OMP_NUM_THREADS", "default (all cores)")}


def run_reference(args, rank, world):
    if rank != 0:
        return
    system = make_system(args.workload if args.workload != "batch" else "chain", args.lmax, args.ncarbon)
    smp = OracleSample(system, args.lmax)
    vals = []
    th = 0.0
    for k in range(args.warmup + args.steps):
        v, th = smp.step()
        if k >= args.warmup:
            vals.append(v)
    v = statistics.median(vals)
    cb = {"value": v, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
          "sample": smp.describe(th) + f"; median of {len(vals)} steps",
          "blas": blas_name(), "blas_threads": os.environ.get("OMP_NUM_THREADS", "default (all cores)")}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
            "higher_is_better": False, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": system.name, "nao": system.basis.nao,
                                            "nocc": system.nocc, "lmax": args.lmax},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# timing helpers (CUDA events on the launching stream, L2 flushed before each)
# ---------------------------------------------------------------------------
class Timer:
    def __init__(self, ctx, dev):
        import torch
        self.torch = torch
        self.ctx = ctx
        self.stream = torch.cuda.current_stream()
        self.flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2

    def run(self, fn, n, warm=2, stages=False):
        """Median ms of n calls (and the mean stage times when asked)."""
        torch = self.torch
        from paper_1708_05353_gb300 import occk
        for _ in range(warm):
            fn()
        ev = []
        st = {k: 0.0 for k in occk.STAGES}
        if stages:
            self.ctx.set_timing(True)
        for k in range(n):
            self.flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(self.stream)
            fn()
            b.record(self.stream)
            ev.append((a, b))
            if stages:
                for s_, v_ in self.ctx.timings().items():
                    st[s_] += v_ / n
        if stages:
            self.ctx.set_timing(False)
        torch.cuda.synchronize()
        ms = statistics.median(a.elapsed_time(b) for a, b in ev)
        return ms, {k: round(v, 4) for k, v in st.items()}


def batch_object(args, dev, steps, prec="fp32", clocks_dev=None):
    """The uneven batch: graphene-like flake, chains of 50/100/200 carbons and
    16 water clusters of 10-60 molecules, lmax 4, in one graph-captured launch
    sequence whose mode and tiles the autotuner picks (level-synchronous
    persistent kernels over all systems, or every system's own pipeline on
    forked streams); timed against the same systems run one call after
    another, and checked against per-system FP64 runs."""
    import numpy as np
    import torch
    from paper_1708_05353_gb300 import inputs, occk
    L = 4
    t0 = time.perf_counter()
    systems = inputs.batch_workload(lmax=L)
    ctx = occk.Context(dev.index or 0)
    trees = []
    for s_ in systems:
        t = occk.Tree(ctx, s_.basis, depth=s_.depth, target_atoms_per_leaf=s_.target_atoms_per_leaf)
        t.pair_multipoles(L)
        trees.append(t)
    b = occk.Batch(ctx, trees, [s_.nocc for s_ in systems], prec=prec)
    for k, s_ in enumerate(systems):
        c, _, _, ld = b.buffers(k)
        occk.device_view(c, (s_.nocc, ld), torch.float64, dev).copy_(torch.tensor(s_.C.T, dtype=torch.float64))
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    cfg = b.tune(args.tune_cache)
    t_tune = time.perf_counter() - t0
    tm = Timer(ctx, dev)
    for _ in range(3):
        b.run(use_graph=True)
    torch.cuda.synchronize()
    clocks = Clocks(clocks_dev) if clocks_dev is not None else None
    ms_graph, _ = tm.run(lambda: b.run(use_graph=True), steps, warm=0)
    clk = clocks.stop() if clocks is not None else None
    ms_nograph, _ = tm.run(lambda: b.run(use_graph=False), steps)
    # both modes at the tuned tile shapes: the level-synchronous persistent
    # kernels over all systems (mode 0) and every system's own pipeline on
    # forked streams (mode 1), each as a captured graph
    modes = {}
    for mode in (0, 1):
        b.set_config(chunk=cfg["chunk"], blocks_per_sm=cfg["blocks_per_sm"], tile=cfg["tile"], mode=mode)
        modes[f"mode{mode}_graph_ms"] = round(tm.run(lambda: b.run(use_graph=True), steps, warm=2)[0], 3)
    b.set_config(**cfg)
    Cs = [occk.fortran(torch.tensor(s_.C, dtype=torch.float64, device=dev)) for s_ in systems]
    Ks = [occk.empty_fortran(s_.basis.nao, s_.nocc, torch.float64, dev) for s_ in systems]
    Es = torch.empty(len(systems), dtype=torch.float64, device=dev)

    def seq():
        for k in range(len(systems)):
            occk.farfield_K(ctx, trees[k], Cs[k], prec=prec, K=Ks[k], Ex=Es[k])
    ms_seq, _ = tm.run(seq, steps)
    Eb = occk.device_view(b.buffers(0)[2], (len(systems),), torch.float64, dev).cpu().numpy()
    for k in range(len(systems)):
        occk.farfield_K(ctx, trees[k], Cs[k], prec="fp64", K=Ks[k], Ex=Es[k])
    torch.cuda.synchronize()
    errs = np.abs(Eb - Es.cpu().numpy())
    out = {"workload": "batch: flake C150H30, chains C50/C100/C200, 16 water clusters 10-60 molecules",
           "nsys": len(systems), "lmax": L, "dtype": "f32" if prec == "fp32" else "f64",
           "tuned": cfg, "tune_s": round(t_tune, 2), "setup_s": round(t_setup, 2),
           "batch_graph_ms": round(ms_graph, 3), "batch_no_graph_ms": round(ms_nograph, 3),
           "sequential_calls_ms": round(ms_seq, 3), "speedup_vs_sequential": round(ms_seq / ms_graph, 3),
           **modes,
           "max_abs_dE_vs_fp64_Eh": float(errs.max()), "clocks": clk}
    del tm
    b.close()
    for t in trees:
        t.close()
    ctx.close()
    return out


def run_batch(args, rank, world, local):
    """`--workload batch`: the batch object as the headline line."""
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = "fp64" if args.prec == "fp64" and args.batch_fp64 else "fp32"
    o = batch_object(args, dev, args.steps, prec=prec, clocks_dev=local)
    ms = max_over_ranks(o["batch_graph_ms"], world, dev)
    line = {"metric": METRIC, "value": ms * 1e-3, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": o["dtype"], "data": "synthetic",
            "config": {"workload": o["workload"], "nsys": o["nsys"], "lmax": o["lmax"], "tuned": o["tuned"],
                       "parallelism": f"replicas x{world}",
                       "l2": "flushed (256 MB write) before every timed step"},
            "clocks": o.pop("clocks"), "batch": o}
    if rank == 0:
        print(json.dumps(line, default=float), flush=True)


def tc_gemm_object(ctx, dev, tm, n=8192):
    """Throughput of the project's tcgen05 GEMM engine (the one steps (a) and
    (e) of the mixed forms use) on a plain n x n x n product D = A B^T from
    FP32 inputs, panel conversion included, per form: the engine's own peak,
    beside cuBLAS's measured BF16 rate (MEASURED_PEAKS.json).  The split forms
    issue three MMAs per product; their rate counts 2 n^3 FLOP once."""
    import torch
    from paper_1708_05353_gb300 import occk
    g = torch.Generator(device="cpu").manual_seed(5)
    A = torch.randn(n, n, generator=g, dtype=torch.float32).to(dev)
    B = torch.randn(n, n, generator=g, dtype=torch.float32).to(dev)
    out = {"shape": [n, n, n], "what": "D = A B^T, FP32 in and out, tcgen05 panel GEMM incl. operand conversion"}
    for prec in ("tf32", "bf16", "fp16", "bf16x3", "fp16x3"):
        ms, _ = tm.run(lambda: occk.debug_tc_gemm(ctx, prec, A, B), 3, warm=1)
        out[prec] = {"ms": round(ms, 3), "tflops": round(2.0 * n ** 3 / (ms * 1e-3) / 1e12, 1)}
    peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks):
        bf = json.load(open(peaks)).get("bf16_tflops")
        if bf:
            out["cublas_bf16_tflops_measured"] = bf
            out["bf16_frac_of_cublas"] = round(out["bf16"]["tflops"] / bf, 3)
    del A, B
    return out


def learned_object(args, ctx, dev, system, tm):
    """The learned per-edge rank selector against fixed rank L_ref (one build
    each; at L_ref = 10 a plain FP64 build of this workload takes about a
    minute and a half), in FP64 and in the split-FP16 form; errors against the
    FP64 build at fixed L_ref."""
    import torch
    from paper_1708_05353_gb300 import learn, occk
    Lr = args.learned_rank
    C = occk.fortran(torch.tensor(system.C, dtype=torch.float64, device=dev))
    K = occk.empty_fortran(system.basis.nao, system.nocc, torch.float64, dev)
    Ex = torch.empty((), dtype=torch.float64, device=dev)
    out = {"lref": Lr, "tau_Eh": args.learned_tau, "what": (
        "FP64 and FP64 from integer slices (fp64s): one build each; split-FP16: one build each after one "
        "untimed call; every form on a context "
        "of its own (the rank-10 workspaces of one form are freed before the next); M2L FLOP ratio from the "
        "chosen ranks, sum_e (L_e+1)^4 vs fixed rank")}
    res = {}
    state = {}

    def one(prec, policy, warm, slices=0):
        # a fresh context and tree per form: FP64 at rank 10 holds ~90 GB of
        # multipoles and local expansions, the tensor-core form its slots and
        # panels; one context with both would not fit
        c2 = occk.Context(ctx.device)
        c2.set_fp64_slices(slices)
        tree = occk.Tree(c2, system.basis, depth=system.depth, target_atoms_per_leaf=system.target_atoms_per_leaf)
        tree.pair_multipoles(Lr)
        learn.load(c2)
        occk.set_learned_tau(c2, args.learned_tau)
        tm2 = Timer(c2, dev)
        try:
            ms, st = tm2.run(lambda: occk.farfield_K(c2, tree, C, prec=prec, lmax_policy=policy, K=K, Ex=Ex), 1,
                             warm=warm, stages=True)
            torch.cuda.synchronize()
            state["ranks"] = occk.edge_ranks(c2, tree) if policy == 2 else None
        finally:
            del tm2
            tree.close()
            c2.close()
            torch.cuda.empty_cache()
        return ms, float(Ex.item()), st

    ms_f, E_f, st_f = one("fp64", 0, 0)
    res["fp64_fixed"] = {"ms": round(ms_f, 2), "E": E_f, "stage_ms": st_f}
    ms_l, E_l, st_l = one("fp64", 2, 0)
    ranks = state["ranks"]
    nedge = len(ranks)
    cost_l = float(((ranks.astype("float64") + 1) ** 4).sum())
    cost_f = float(nedge * (Lr + 1) ** 4)
    res["fp64_learned"] = {"ms": round(ms_l, 2), "abs_dE_vs_fixed_fp64_Eh": abs(E_l - E_f),
                           "speedup_vs_fixed_fp64": round(ms_f / ms_l, 3),
                           "m2l_flop_ratio_fixed_over_learned": round(cost_f / max(cost_l, 1.0), 3),
                           "rank_histogram": [int(x) for x in
                                              __import__("numpy").bincount(ranks, minlength=Lr + 1)],
                           "stage_ms": st_l}
    # the FP64-accurate form from integer slices and double-FP32 arithmetic
    ms_sf, E_sf, st_sf = one("fp64", 0, 0, slices=7)
    res["fp64s_fixed"] = {"ms": round(ms_sf, 2), "abs_dE_vs_fixed_fp64_Eh": abs(E_sf - E_f),
                          "speedup_vs_fixed_fp64": round(ms_f / ms_sf, 3), "stage_ms": st_sf}
    ms_sl, E_sl, st_sl = one("fp64", 2, 0, slices=7)
    res["fp64s_learned"] = {"ms": round(ms_sl, 2), "abs_dE_vs_fixed_fp64_Eh": abs(E_sl - E_f),
                            "abs_dE_vs_fp64_learned_Eh": abs(E_sl - E_l),
                            "speedup_vs_fixed_fp64": round(ms_f / ms_sl, 3),
                            "speedup_vs_fixed_fp64s": round(ms_sf / ms_sl, 3), "stage_ms": st_sl}
    ms_hf, E_hf, _ = one("fp16x3", 0, 1)
    res["fp16x3_fixed"] = {"ms": round(ms_hf, 2), "abs_dE_vs_fixed_fp64_Eh": abs(E_hf - E_f),
                           "speedup_vs_fixed_fp64": round(ms_f / ms_hf, 3)}
    ms_hl, E_hl, st_hl = one("fp16x3", 2, 1)
    res["fp16x3_learned"] = {"ms": round(ms_hl, 2), "abs_dE_vs_fixed_fp64_Eh": abs(E_hl - E_f),
                             "speedup_vs_fixed_fp64": round(ms_f / ms_hl, 3), "stage_ms": st_hl}
    out.update(res)
    return out


def chain_object(args, ctx, dev, tm):
    """C150H302 at rank 2: FP64 from integer slices, FP32 (SIMT) and FP16X3
    (tensor core), against the FP64 GPU form and the oracle's exact columns."""
    import torch
    from paper_1708_05353_gb300 import occk
    s = make_system("chain", 2, args.ncarbon)
    tree = occk.Tree(ctx, s.basis, depth=s.depth, target_atoms_per_leaf=s.target_atoms_per_leaf)
    tree.pair_multipoles(2)
    C = occk.fortran(torch.tensor(s.C, dtype=torch.float64, device=dev))
    K = occk.empty_fortran(s.basis.nao, s.nocc, torch.float64, dev)
    Ex = torch.empty((), dtype=torch.float64, device=dev)
    gold = golden_columns("chain", 2, s)
    out = {"workload": s.name, "nao": s.basis.nao, "nocc": s.nocc, "lmax": 2, "depth": tree.info()["depth"]}
    n = max(5, args.steps // 2)
    ms64, _ = tm.run(lambda: occk.farfield_K(ctx, tree, C, prec="fp64", K=K, Ex=Ex), max(3, n // 2))
    E64 = float(Ex.item())
    K64 = K.clone()
    out["fp64"] = {"ms": round(ms64, 4), "E": E64, **oracle_errors(gold, K64, s.C)}
    for p in ("fp64s", "fp32", "fp16x3"):
        ctx.set_fp64_slices(SLICED.get(p, 0))
        try:
            ms, st = tm.run(lambda: occk.farfield_K(ctx, tree, C, prec="fp64" if p in SLICED else p, K=K, Ex=Ex), n,
                            stages=True)
        finally:
            ctx.set_fp64_slices(0)
        out[p] = {"ms": round(ms, 4), "speedup_vs_fp64": round(ms64 / ms, 3),
                  "abs_dE_vs_fp64_Eh": abs(float(Ex.item()) - E64),
                  "rel_dK_vs_fp64": float((K - K64).abs().max() / K64.abs().max()),
                  **oracle_errors(gold, K, s.C), "stage_ms": st}
    tree.close()
    return out


def screen_object(args, ctx, dev, tm):
    """Occupied-pair screening on the localised orbitals of C150H302 (same
    geometry, basis and tree as the chain): unscreened and screened, FP32 and
    FP16X3."""
    import torch
    from paper_1708_05353_gb300 import occk
    sl = make_system("chain-loc", 2, args.ncarbon)
    tree = occk.Tree(ctx, sl.basis, depth=sl.depth, target_atoms_per_leaf=sl.target_atoms_per_leaf)
    tree.pair_multipoles(2)
    Cl = occk.fortran(torch.tensor(sl.C, dtype=torch.float64, device=dev))
    K = occk.empty_fortran(sl.basis.nao, sl.nocc, torch.float64, dev)
    Ex = torch.empty((), dtype=torch.float64, device=dev)
    n = max(5, args.steps // 2)

    def timed(tau, prec):
        ctx.set_pair_screen(tau)
        try:
            ms, st = tm.run(lambda: occk.farfield_K(ctx, tree, Cl, prec=prec, K=K, Ex=Ex), n, stages=True)
            kept = ctx.pair_screen_count()
        finally:
            ctx.set_pair_screen(0.0)
        return ms, float(Ex.item()), K.clone(), kept, st

    E64 = timed(0.0, "fp64")[1]
    npair = sl.nocc * (sl.nocc + 1) // 2
    out = {"workload": sl.name + " (same geometry, basis and tree as the chain; localised occupied orbitals)",
           "tau": args.screen_tau, "pairs": npair}
    for p in ("fp32", "fp16x3"):
        ms0, E0, K0, _, st0 = timed(0.0, p)
        ms1, E1, K1, kept, st1 = timed(args.screen_tau, p)
        out[p] = {"ms_unscreened": round(ms0, 4), "ms_screened": round(ms1, 4), "speedup": round(ms0 / ms1, 3),
                  "kept_pairs": kept, "kept_fraction": round(kept / npair, 4),
                  "abs_dE_screened_vs_unscreened_Eh": abs(E1 - E0),
                  "abs_dE_screened_vs_fp64_unscreened_Eh": abs(E1 - E64),
                  "rel_dK": float((K1 - K0).abs().max() / K0.abs().max()),
                  "stage_ms_unscreened": st0, "stage_ms_screened": st1}
    tree.close()
    return out


def main(argv=None):
    args = parse(argv)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1708_05353_gb300 import occk, shard

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    if args.workload == "batch":
        run_batch(args, rank, world, local)
        return
    t_in = time.perf_counter()
    system = make_system(args.workload, args.lmax, args.ncarbon)
    t_in = time.perf_counter() - t_in
    L = args.lmax
    ctx = occk.Context(local)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    # set-up, reported apart from the timed builds: the host tree and step a0
    # (pair multipoles and operators on the device), wall clock, first call
    t_set0 = time.perf_counter()
    tree = occk.Tree(ctx, system.basis, depth=system.depth, target_atoms_per_leaf=system.target_atoms_per_leaf)
    t_tree = time.perf_counter() - t_set0
    info = tree.info()
    torch.cuda.synchronize()
    t_set0 = time.perf_counter()
    tree.pair_multipoles(L)
    torch.cuda.synchronize()
    t_a0 = time.perf_counter() - t_set0
    C = torch.tensor(system.C, dtype=torch.float64, device=dev)
    Cf = occk.fortran(C)
    K = occk.empty_fortran(system.basis.nao, system.nocc, torch.float64, dev)
    Ex = torch.empty((), dtype=torch.float64, device=dev)
    tm = Timer(ctx, dev)
    stream = tm.stream
    blocks = shard.column_blocks(system.nocc, world)
    col0, col1 = blocks[rank]

    if args.workload == "chain-loc":
        ctx.set_pair_screen(args.screen_tau)     # every build below is screened
    if args.fp64_slices and args.prec == "fp64":
        ctx.set_fp64_slices(args.fp64_slices)    # the main line and e2e; variants reset it

    def step():
        if world > 1:
            shard.farfield_K_sharded(ctx, tree, Cf, blocks, rank, prec=args.prec, K=K, Ex=Ex)
        else:
            occk.farfield_K(ctx, tree, Cf, prec=args.prec, K=K, Ex=Ex)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # FMA peak of this GPU, measured now and again after the timed region
    probe0 = ctx.probe_fma_peak("fp64" if args.prec == "fp64" else "fp32")

    # ---- timed region: K steps, L2 flushed before each, events around each
    ctx.set_timing(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    stage_ms = {k: 0.0 for k in occk.STAGES}
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        tm.flush.fill_(float(k))
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
        for n, v in ctx.timings().items():
            stage_ms[n] += v
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ctx.set_timing(False)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = statistics.median(step_ms)
    stage_ms = {k: v / args.steps for k, v in stage_ms.items()}
    ms_max = max_over_ranks(ms, world, dev)
    E_main = float(Ex.item())
    K_main = K.clone()

    # ---- end-to-end: host C (pinned) -> device -> K, E back to host
    Ch = torch.tensor(system.C.T.copy(), dtype=torch.float64).pin_memory()   # [nocc, nao] = column-major C
    Kh = torch.empty((system.nocc, system.basis.nao), dtype=torch.float64).pin_memory()
    Eh = torch.empty((), dtype=torch.float64).pin_memory()
    Cd = torch.empty((system.nocc, system.basis.nao), dtype=torch.float64, device=dev)
    n_e2e = max(3, min(args.steps, 5))

    def e2e_step():
        Cd.copy_(Ch, non_blocking=True)
        if world > 1:
            shard.farfield_K_sharded(ctx, tree, Cd.t(), blocks, rank, prec=args.prec, K=K, Ex=Ex)
        else:
            occk.farfield_K(ctx, tree, Cd.t(), prec=args.prec, K=K, Ex=Ex)
        Kh.copy_(K.t(), non_blocking=True)
        Eh.copy_(Ex, non_blocking=True)
    e2e_ms, _ = tm.run(e2e_step, n_e2e, warm=1)
    e2e_max = max_over_ranks(e2e_ms, world, dev)

    # ---- roofline of the dominant kernel against the measured FMA peak
    lo = tree.export("level_off")
    D = info["depth"]
    nm2m = int(lo[D + 1] - lo[3]) if D >= 3 else 0
    rowoff = tree.export("leaf_rowoff")
    flops = stage_flops(rowoff, system.nocc, L, info["nentry"], nm2m, nm2m, info["nm2l"])
    total_flops = sum(flops.values())
    # the SIMT path runs M2L and L2L as one pass per level: the L2L stage
    # then has no time of its own and its FLOPs belong to the fused stage
    fused_cd = D >= 3 and stage_ms["d_l2l"] < 0.01 * stage_ms["c_m2l"]
    fl = dict(flops)
    if fused_cd or D < 3:
        fl["c_m2l"] += fl["d_l2l"]
        fl["d_l2l"] = 0.0
    dom = max(stage_ms, key=lambda k: stage_ms[k])
    peak_prec = "fp64" if args.prec == "fp64" else "fp32"
    probe = max(probe0, ctx.probe_fma_peak(peak_prec))
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    nominal = (1.25e12 * sm_count / 152.0 if peak_prec == "fp64" else sm_count * 128 * 2 * 2.07e9) * sm_mhz / 2070.0
    kernel_names = {"a_half": "k_half", "a_full": "k_full", "b_m2m": "k_translate(M2M)",
                    "c_m2l": "k_translate(M2L+L2L)" if fused_cd else "k_translate(M2L)",
                    "d_l2l": "k_translate(L2L)", "e_l2p": "k_l2p_r32" if args.prec == "fp64" else "k_l2p",
                    "reduce": "k_reduce_K"}
    sliced_m2l = bool(args.fp64_slices) and args.prec == "fp64" and (L + 1) ** 2 >= 25
    if args.fp64_slices and args.prec == "fp64":
        kernel_names.update({"a_half": "k_half_ff", "a_full": "k_s_gemm_a", "b_m2m": "k_translate_ff(M2M)",
                             "c_m2l": ("k_s_gemm_m2l(M2L)+k_translate_ff(L2L)" if sliced_m2l
                                       else "k_translate_ff(M2L+L2L)"),
                             "e_l2p": "k_s_gemm_e"})
    achieved = fl[dom] / (stage_ms[dom] * 1e-3)
    bound = "alu"
    peak_source = (f"measured: independent-accumulator {peak_prec.upper()} FMA probe "
                   f"(occk_probe_fma_peak) on this GPU in this run, {probe / 1e12:.3f} TFLOP/s; nominal "
                   f"{sm_count} SMs at the median {sm_mhz:.0f} MHz: {nominal / 1e12:.3f} TFLOP/s")
    if args.fp64_slices and args.prec == "fp64":
        if dom in ("a_full", "e_l2p") or (dom == "c_m2l" and sliced_m2l):
            # slice GEMM: S (S + 1) / 2 FP16 products per FP64 product, against
            # the dense 16-bit tensor rate measured with cuBLAS on this machine
            npr = args.fp64_slices * (args.fp64_slices + 1) // 2
            bf = None
            try:
                bf = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("bf16_tflops")
            except Exception:
                pass
            bf = (bf or 1900.0) * 1e12
            bound, achieved, probe, nominal = "tensor", achieved * npr, bf, 2.25e15
            peak_source = (f"measured cuBLAS dense BF16 rate of this pool (FP16 runs at the same rate), "
                           f"{bf / 1e12:.0f} TFLOP/s; achieved counts the {npr} slice products of each "
                           f"FP64 multiply-add")
        elif dom in ("a_half", "b_m2m", "c_m2l"):
            # double-FP32 pass: 12 FP32 operations per FP64-equivalent
            # multiply-add (error-free product 4, TwoSum 6, error folding 2)
            p32 = ctx.probe_fma_peak("fp32")
            probe, nominal = p32 / 12.0, sm_count * 128 * 2 * 2.07e9 * sm_mhz / 2070.0 / 12.0
            peak_source = (f"measured FP32 FMA probe (occk_probe_fma_peak) in this run, {p32 / 1e12:.2f} "
                           f"TFLOP/s, / 12 FP32 operations per double-FP32 multiply-add = "
                           f"{probe / 1e12:.3f} TFLOP/s of FP64-equivalent work")
    roof = {"bound": bound, "kernel": kernel_names[dom], "stage": dom,
            "achieved": achieved / 1e12, "peak": probe / 1e12, "unit": "TFLOP/s",
            "frac": achieved / probe, "traffic": traffic_for(kernel_names[dom]),
            "peak_source": peak_source,
            "frac_of_nominal": achieved / nominal,
            "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
            "stage_tflops": {k: round(fl[k] / max(stage_ms[k], 1e-9) / 1e9, 4) for k in fl}}

    # transpose, half, full, D-2 M2M, D-1 fused M2L+L2L, L2P, reduction,
    # energy; screened FP32/FP64 builds add the two step (a) bound kernels and
    # part, flag, scan, compact, tiles, gather and scatter
    nlaunch = 7 + 2 * max(D - 2, 0) + (9 if args.workload == "chain-loc" else 0)
    result = {
        "metric": METRIC,
        "value": job_seconds_per_build(ms_max, world),
        "unit": "s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max,
        "higher_is_better": False,
        "scaling": "strong",
        "vs_baseline": None,
        "dtype": "f64" if args.prec == "fp64" else args.prec,
        "data": "synthetic",
        "config": {"workload": system.name + (f", occupied pairs screened at tau {args.screen_tau:g}"
                                              if args.workload == "chain-loc" else ""),
                   "nao": system.basis.nao, "nocc": system.nocc,
                   "lmax": L, "depth": D, "nbox": info["nbox"], "nm2l": info["nm2l"],
                   "precision": args.prec + (f" (steps a, e from {args.fp64_slices} integer slices on the tensor "
                                             "core; half transform and tree passes in double-FP32)"
                                             if args.fp64_slices and args.prec == "fp64" else ""),
                   "parallelism": (f"occupied column blocks x{world} (gathered over NCCL)" if world > 1
                                   else "one GPU"),
                   "l2": "flushed (256 MB write) before every timed step",
                   "timing": "median of the timed steps (CUDA events on the launch stream)"},
        "tflops": total_flops / (ms_max * 1e-3) / 1e12,
        "algorithmic_gflop_per_step": total_flops / 1e9,
        "wall_s_timed_region": t_wall,
        "step_ms_min_max": [min(step_ms), max(step_ms)],
        "e2e": {"value": job_seconds_per_build(e2e_max, world), "unit": "s",
                "h2d_bytes_per_step": int(system.basis.nao * system.nocc * 8),
                "d2h_bytes_per_step": int(system.basis.nao * system.nocc * 8 + 8),
                "steps": n_e2e},
        "gpu_launches": nlaunch * args.steps,
        "roofline": roof,
        "clocks": clk,
        "energy": E_main,
        "setup": {"inputs_s": round(t_in, 2), "build_tree_s": round(t_tree, 4),
                  "pair_multipoles_s": round(t_a0, 4),
                  "what": "input generation (host), host tree and step a0 on the device, wall clock, "
                          "first call, outside the timed region"},
    }
    gold = golden_columns(args.workload, L, system) if world == 1 else None
    if gold is not None:
        result["error_vs_oracle"] = oracle_errors(gold, K_main, system.C)
        result["error_vs_oracle"]["what"] = ("exact oracle K columns (tests/golden/oracle_columns.npz, "
                                             "written from the FP64 oracle alone)")
    if rank == 0 and world == 1:
        # ---- the mixed forms on the same workload: time, speed-up over the
        # FP64 GPU form, error against it and against the oracle's columns
        ctx.set_fp64_slices(0)
        if args.variants != "none":
            if args.prec == "fp64" and not args.fp64_slices:
                ms64, E64, K64 = ms_max, E_main, K_main
            else:
                ms64, _ = tm.run(lambda: occk.farfield_K(ctx, tree, Cf, prec="fp64", K=K, Ex=Ex), 3, warm=1)
                E64, K64 = float(Ex.item()), K.clone()
            kmax = float(K64.abs().max())
            var = {}
            for vp in [v for v in args.variants.split(",") if v and v != args.prec]:
                ctx.set_fp64_slices(SLICED.get(vp, 0))
                ctx.set_fp32_slices(F32SLICED.get(vp, 0))
                vprec = "fp64" if vp in SLICED else "fp32" if vp in F32SLICED else vp
                try:
                    vms, vst = tm.run(lambda: occk.farfield_K(ctx, tree, Cf, prec=vprec, K=K, Ex=Ex),
                                      max(5, args.steps // 2), stages=True)
                finally:
                    ctx.set_fp64_slices(0)
                    ctx.set_fp32_slices(0)
                var[vp] = {"ms": round(vms, 4), "speedup_vs_fp64": round(ms64 / vms, 3),
                           "tflops": round(total_flops / (vms * 1e-3) / 1e12, 3),
                           "abs_dE_vs_fp64_Eh": abs(float(Ex.item()) - E64),
                           "rel_dK_vs_fp64": float((K - K64).abs().max()) / kmax,
                           **oracle_errors(gold, K, system.C),
                           "stage_ms": vst}
            result["variants"] = var
            result["variants_reference"] = ("speed-up and errors against the FP64 GPU form of the same run "
                                            f"({ms64:.2f} ms, E = {E64:.10f} Eh), which matches the oracle's "
                                            "columns to the stated error; fp64s / fp64s6: FP64 with steps (a) "
                                            "and (e) from 7 / 6 integer slices on the tensor core and the other "
                                            "passes in double-FP32; fp32s: FP32 with steps (a) and (e) from 4 "
                                            "integer slices (tflops: FLOPs of the algorithm per second)")
        if args.workload == "protein" and args.learned_rank > 0:
            try:
                result["learned"] = learned_object(args, ctx, dev, system, tm)
            except Exception as ex:      # reported, not fatal for the main line
                result["learned"] = {"error": repr(ex)}
        if args.workload == "protein" and not args.no_chain:
            try:
                result["chain"] = chain_object(args, ctx, dev, tm)
            except Exception as ex:
                result["chain"] = {"error": repr(ex)}
        # ---- far-field Coulomb matrix on the same tree and rank (FP64),
        # density D = 2 C C^T made outside the timed region
        try:
            Dm = occk.fortran(2.0 * C @ C.t())
            J = occk.empty_fortran(system.basis.nao, system.basis.nao, torch.float64, dev)
            Ej = torch.empty((), dtype=torch.float64, device=dev)
            jms, _ = tm.run(lambda: occk.farfield_J(ctx, tree, Dm, J=J, Ej=Ej), max(3, args.steps // 2), warm=3)
            result["coulomb_j"] = {"ms": round(jms, 4), "E_J": float(Ej.item()), "lmax": L, "dtype": "f64",
                                   "what": "far-field J^ff and E_J on the same tree, D = 2 C C^T"}
            del Dm, J
        except Exception as ex:
            result["coulomb_j"] = {"error": repr(ex)}
        if args.workload == "protein":
            try:
                result["tc_gemm"] = tc_gemm_object(ctx, dev, tm)
            except Exception as ex:
                result["tc_gemm"] = {"error": repr(ex)}
        if args.workload == "protein" and not args.no_batch:
            try:
                result["batch"] = batch_object(args, dev, max(5, args.steps // 2))
            except Exception as ex:
                result["batch"] = {"error": repr(ex)}
        if args.screen_tau > 0 and args.workload in ("protein", "chain"):
            try:
                result["pair_screen"] = screen_object(args, ctx, dev, tm)
            except Exception as ex:
                result["pair_screen"] = {"error": repr(ex)}
        if not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline(system, L)
    if rank == 0:
        print(json.dumps(result, default=float), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
