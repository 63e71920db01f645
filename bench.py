#!/usr/bin/env python
"""Benchmark of the far-field occ-FMM-K exchange build on GB300.

Workload (default): the 150-carbon zig-zag alkane chain C150H302 with the
synthetic s/p basis (C: 2s1p, H: 2s, 3 primitives, log-uniform exponents in
[0.1, 50]), 1354 AOs, nocc = 601 Loewdin-orthonormalised random orbitals,
octree to ~8 atoms per leaf (depth 6), lmax = 2, FP32 contractions.  One
"step" = one occk_farfield_K call (steps a-e: C on the device -> K^ff, E^ff).

Prints ONE JSON line on rank 0.  `value` = seconds per far-field K build for
the whole job (lower is better); with N GPUs each rank builds its own replica
(replicas only, weak scaling).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("far-field K_ri build time (s) & TFLOP/s at stated error vs FP64 oracle, "
          "learned/mixed vs plain")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--ncarbon", type=int, default=150)
    p.add_argument("--lmax", type=int, default=2)
    p.add_argument("--prec", default="fp32",
                   help="main precision; the C150H302 workload is specified for plain FP64/FP32")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-cols", type=int, default=2)
    p.add_argument("--workload", default="chain", choices=["chain", "chain-loc", "water", "batch"],
                   help="chain-loc: the chain with localised orbitals, every build screened at --screen-tau")
    p.add_argument("--batch-fp64", action="store_true", help="run the batch workload in FP64 (default FP32)")
    p.add_argument("--screen-tau", type=float, default=1e-4,
                   help="occupied-pair screening threshold timed on localised orbitals of the same chain "
                        "(0: skip)")
    p.add_argument("--variants", default="fp64,fp32,tf32,bf16,fp16,bf16x3,fp16x3",
                   help="extra precisions timed beside the main one (comma list, or 'none')")
    return p.parse_args()


def make_system(args):
    from paper_1708_05353_gb300 import inputs
    if args.workload == "water":
        return inputs.water(100, lmax=args.lmax)
    if args.workload == "chain-loc":
        return inputs.alkane_localised(args.ncarbon, lmax=args.lmax)
    return inputs.alkane(args.ncarbon, lmax=args.lmax)


# ---------------------------------------------------------------------------
# algorithmic FLOPs per stage (real form; only the symmetric half of the
# occupied pairs in (a) O^{ij} and in the tree passes b-d)
# ---------------------------------------------------------------------------
def stage_flops(tree_info, rowoff, nocc, L, depth, level_off, nent, nm2m, nl2l, nm2l):
    nc = (L + 1) ** 2
    tl = sum((2 * l + 1) * (l + 1) ** 2 for l in range(L + 1))
    P = nocc * (nocc + 1) // 2          # the tree passes need only pairs i <= j
    S = [rowoff[k + 1] - rowoff[k] for k in range(len(rowoff) - 1)]
    return {
        "a_half": 2.0 * nent * nocc * nc,
        "a_full": sum(2.0 * s * nc * nocc * (nocc + 1) / 2 for s in S),
        "b_m2m": 2.0 * tl * P * nm2m,
        "c_m2l": 2.0 * nc * nc * P * nm2l,
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
    """Whole-job time per far-field K build: each of `world` replicas builds
    one K per step, and the slowest rank's step time is ms_max."""
    return ms_max * 1e-3 / world


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


def cpu_baseline(system, L, ncols):
    """The FP64 oracle, as it stands, on a bounded sample: all of step a0 and
    the AO->MO half transform, plus K for `ncols` occupied columns; the full
    build time is extrapolated linearly in the number of columns."""
    import numpy as np
    from oracle import fmm
    from oracle import tree as otree
    t0 = time.perf_counter()
    tr = otree.build_tree(system.basis, system.depth, system.target_atoms_per_leaf)
    Op = fmm.pair_multipoles(system.basis, tr, L)
    W = fmm.half_transform(system.basis, tr, Op, system.C, L)
    t1 = time.perf_counter()
    cols = list(range(ncols))
    fmm.farfield(system, L=L, tree=tr, i_subset=cols, Opair=Op, W=W)
    t2 = time.perf_counter()
    t_cols = t2 - t1
    est = (t1 - t0) + t_cols * system.nocc / ncols
    del W, Op
    return {"value": est, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"oracle FP64 on {system.name} L={L}: tree + pair multipoles + half transform "
                       f"({t1 - t0:.1f} s) and K for {ncols} of {system.nocc} columns "
                       f"({t_cols:.1f} s), extrapolated linearly to all columns"),
            "blas_threads": os.environ.get("OMP_NUM_THREADS", "default")}


def run_reference(args, rank, world):
    if rank != 0:
        return
    system = make_system(args)
    vals = []
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(system, args.lmax, args.cpu_cols)
        if k >= args.warmup:
            vals.append(cb["value"])
    v = statistics.median(vals)
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": system.name, "nao": system.basis.nao,
                                            "nocc": system.nocc, "lmax": args.lmax},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args, rank, world, local):
    """The uneven batch: graphene-like flake, chains of 50/100/200 carbons and
    16 water clusters of 10-60 molecules, lmax 4, FP32 contractions, in one
    persistent, graph-captured launch sequence with autotuned tiles; timed
    against the same systems run one call after another."""
    import torch
    from paper_1708_05353_gb300 import inputs, occk
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    L = 4
    systems = inputs.batch_workload(lmax=L)
    ctx = occk.Context(local)
    trees = []
    for s_ in systems:
        t = occk.Tree(ctx, s_.basis, depth=s_.depth, target_atoms_per_leaf=s_.target_atoms_per_leaf)
        t.pair_multipoles(L)
        trees.append(t)
    prec = "fp64" if args.prec == "fp64" and args.batch_fp64 else "fp32"
    b = occk.Batch(ctx, trees, [s_.nocc for s_ in systems], prec=prec)
    for k, s_ in enumerate(systems):
        c, _, _, ld = b.buffers(k)
        occk.device_view(c, (s_.nocc, ld), torch.float64, dev).copy_(torch.tensor(s_.C.T, dtype=torch.float64))
    cfg = b.tune(os.path.join(ROOT, "profiles", "batch_tune_cache.txt"))
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def timed(fn, n):
        ev = []
        for k in range(n):
            flush.fill_(float(k))
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            e.record(stream)
            ev.append((a, e))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(e) for a, e in ev) / n

    for _ in range(max(args.warmup, 3)):
        b.run(use_graph=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    ms_graph = timed(lambda: b.run(use_graph=True), args.steps)
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms_graph = max_over_ranks(ms_graph, world, dev)
    ms_nograph = timed(lambda: b.run(use_graph=False), args.steps)
    Cs = [occk.fortran(torch.tensor(s_.C, dtype=torch.float64, device=dev)) for s_ in systems]
    Ks = [occk.empty_fortran(s_.basis.nao, s_.nocc, torch.float64, dev) for s_ in systems]
    Es = torch.empty(len(systems), dtype=torch.float64, device=dev)

    def seq():
        for k in range(len(systems)):
            occk.farfield_K(ctx, trees[k], Cs[k], prec=prec, K=Ks[k], Ex=Es[k])
    for _ in range(2):
        seq()
    ms_seq = timed(seq, args.steps)
    # errors of the batch against per-system FP64 runs
    import numpy as np
    Eb = occk.device_view(b.buffers(0)[2], (len(systems),), torch.float64, dev).cpu().numpy()
    errs = []
    for k in range(len(systems)):
        occk.farfield_K(ctx, trees[k], Cs[k], prec="fp64", K=Ks[k], Ex=Es[k])
    torch.cuda.synchronize()
    E64 = Es.cpu().numpy()
    errs = np.abs(Eb - E64)
    line = {"metric": METRIC, "value": job_seconds_per_build(ms_graph, world), "unit": "s", "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": "batch: flake C150H30, chains C50/C100/C200, 16 water clusters 10-60",
                       "nsys": len(systems), "lmax": L, "tuned": cfg,
                       "l2": "flushed (256 MB write) before every timed step"},
            "batch_graph_ms": ms_graph, "batch_no_graph_ms": ms_nograph, "sequential_calls_ms": ms_seq,
            "speedup_vs_sequential": ms_seq / ms_graph, "max_abs_dE_vs_fp64_Eh": float(errs.max()),
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line, default=float), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1708_05353_gb300 import inputs, occk

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    if args.workload == "batch":
        run_batch(args, rank, world, local)
        return
    system = make_system(args)
    L = args.lmax
    ctx = occk.Context(local)
    # set-up, reported apart from the timed builds: the host tree and step a0
    # (pair multipoles and operators on the device), wall clock, first call
    t_set0 = time.perf_counter()
    tree = occk.Tree(ctx, system.basis, depth=system.depth,
                     target_atoms_per_leaf=system.target_atoms_per_leaf)
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
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream()

    if args.workload == "chain-loc":
        ctx.set_pair_screen(args.screen_tau)     # every build below is screened

    def step():
        occk.farfield_K(ctx, tree, Cf, prec=args.prec, K=K, Ex=Ex)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

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
        flush.fill_(float(k))
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
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    stage_ms = {k: v / args.steps for k, v in stage_ms.items()}
    ms_max = max_over_ranks(ms, world, dev)

    # ---- end-to-end: host C (pinned) -> device -> K, E back to host
    Ch = torch.tensor(system.C.T.copy(), dtype=torch.float64).pin_memory()   # [nocc, nao] = column-major C
    Kh = torch.empty((system.nocc, system.basis.nao), dtype=torch.float64).pin_memory()
    Eh = torch.empty((), dtype=torch.float64).pin_memory()
    Cd = torch.empty((system.nocc, system.basis.nao), dtype=torch.float64, device=dev)
    e2e_ev = []
    for k in range(args.warmup + args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        Cd.copy_(Ch, non_blocking=True)
        occk.farfield_K(ctx, tree, Cd.t(), prec=args.prec, K=K, Ex=Ex)
        Kh.copy_(K.t(), non_blocking=True)
        Eh.copy_(Ex, non_blocking=True)
        b.record(stream)
        if k >= args.warmup:
            e2e_ev.append((a, b))
    torch.cuda.synchronize()
    e2e_ms = sum(a.elapsed_time(b) for a, b in e2e_ev) / len(e2e_ev)
    e2e_max = max_over_ranks(e2e_ms, world, dev)

    # ---- roofline of the dominant kernel
    lo = tree.export("level_off")
    D = info["depth"]
    nm2m = int(lo[D + 1] - lo[3]) if D >= 3 else 0
    flops = stage_flops(info, tree.export("leaf_rowoff"), system.nocc, L, D, lo, info["nentry"],
                        nm2m, nm2m, info["nm2l"])
    total_flops = sum(flops.values())
    # the SIMT path runs M2L and L2L as one pass per level: the L2L stage
    # then has no time of its own and its FLOPs belong to the fused stage
    fused_cd = D >= 3 and stage_ms["d_l2l"] < 0.01 * stage_ms["c_m2l"]
    if fused_cd:
        flops["c_m2l"] += flops["d_l2l"]
        flops["d_l2l"] = 0.0
    dom = max(stage_ms, key=lambda k: stage_ms[k])
    peak_prec = "fp64" if args.prec == "fp64" else "fp32"
    probe = ctx.probe_fma_peak(peak_prec)
    # nominal unit rates at the maximum SM clock (2070 MHz): FP64 1.25 TFLOP/s
    # (2 DFMA/clk/SM), FP32 152 SMs x 128 FFMA/clk x 2; scaled by the median SM
    # clock sampled during the timed region
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    nominal = 1.25e12 if peak_prec == "fp64" else 152 * 128 * 2 * 2.07e9
    peak = nominal * sm_mhz / 2070.0
    kernel_names = {"a_half": "k_half", "a_full": "k_full", "b_m2m": "k_translate(M2M)",
                    "c_m2l": "k_translate(M2L+L2L)" if fused_cd else "k_translate(M2L)",
                    "d_l2l": "k_translate(L2L)", "e_l2p": "k_l2p",
                    "reduce": "k_reduce_K"}
    achieved = flops[dom] / (stage_ms[dom] * 1e-3)
    roof = {"bound": "alu", "kernel": kernel_names[dom], "stage": dom,
            "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic_for(kernel_names[dom]),
            "peak_source": (f"nominal {peak_prec.upper()} rate scaled to the median SM clock "
                            f"({sm_mhz:.0f} MHz); a dependent-FMA probe measured {probe / 1e12:.3f} TFLOP/s"),
            "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
            "stage_tflops": {k: round(flops[k] / max(stage_ms[k], 1e-9) / 1e9, 4) for k in flops}}

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
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.prec == "fp64" else args.prec,
        "data": "synthetic",
        "config": {"workload": system.name + (f", occupied pairs screened at tau {args.screen_tau:g}"
                                              if args.workload == "chain-loc" else ""),
                   "nao": system.basis.nao, "nocc": system.nocc,
                   "lmax": L, "depth": D, "nbox": info["nbox"], "nm2l": info["nm2l"],
                   "precision": args.prec, "parallelism": f"replicas x{world}",
                   "l2": "flushed (256 MB write) before every timed step"},
        "tflops": total_flops * world / (ms_max * 1e-3) / 1e12,     # whole job (replicas)
        "algorithmic_gflop_per_step": total_flops / 1e9,
        "wall_s_timed_region": t_wall,
        "e2e": {"value": job_seconds_per_build(e2e_max, world), "unit": "s",
                "h2d_bytes_per_step": int(system.basis.nao * system.nocc * 8),
                "d2h_bytes_per_step": int(system.basis.nao * system.nocc * 8 + 8)},
        "gpu_launches": nlaunch * args.steps,
        "roofline": roof,
        "clocks": clk,
        "energy": float(Ex.item()),
        "setup": {"build_tree_s": round(t_tree, 4), "pair_multipoles_s": round(t_a0, 4),
                  "what": "host tree and step a0 on the device, wall clock, first call, outside the timed region"},
    }
    # ---- other precisions on the same workload: time and error against the
    # FP64 GPU result (which the parity tests tie to the FP64 oracle)
    if args.variants != "none":
        E64 = None
        K64 = None
        if args.prec == "fp64":
            E64 = float(Ex.item())
            K64 = K.clone()
        else:
            Kmain, Emain = K.clone(), float(Ex.item())
            occk.farfield_K(ctx, tree, Cf, prec="fp64", K=K, Ex=Ex)
            E64 = float(Ex.item())
            K64 = K.clone()
        kmax = float(K64.abs().max().item())
        if args.prec != "fp64":
            result["error_vs_fp64"] = {"abs_dE_Eh": abs(Emain - E64),
                                       "rel_dK": float((Kmain - K64).abs().max().item()) / kmax}
        var = {}
        for vp in [v for v in args.variants.split(",") if v and v != args.prec]:
            for _ in range(2):
                occk.farfield_K(ctx, tree, Cf, prec=vp, K=K, Ex=Ex)
            ev = []
            vst = {k: 0.0 for k in occk.STAGES}
            ctx.set_timing(True)
            nv = max(3, args.steps // 2)
            for k in range(nv):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                occk.farfield_K(ctx, tree, Cf, prec=vp, K=K, Ex=Ex)
                b.record(stream)
                ev.append((a, b))
                for n_, v_ in ctx.timings().items():
                    vst[n_] += v_ / nv
            ctx.set_timing(False)
            torch.cuda.synchronize()
            vms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
            var[vp] = {"ms": round(vms, 4), "speedup_vs_fp64": round(ms_max / vms, 3) if args.prec == "fp64" else None,
                       "tflops": round(total_flops / (vms * 1e-3) / 1e12, 3),
                       "abs_dE_Eh": abs(float(Ex.item()) - E64),
                       "rel_dK": float((K - K64).abs().max().item()) / kmax,
                       "stage_ms": {k: round(v, 4) for k, v in vst.items()}}
        result["variants"] = var
        result["variants_reference"] = "errors against the FP64 GPU path of the same run (E = %.10f Eh)" % E64
    # ---- far-field Coulomb matrix on the same tree and rank (FP64), density
    # D = 2 C C^T made outside the timed region
    Dm = occk.fortran(2.0 * C @ C.t())
    J = occk.empty_fortran(system.basis.nao, system.basis.nao, torch.float64, dev)
    Ej = torch.empty((), dtype=torch.float64, device=dev)
    for _ in range(3):
        occk.farfield_J(ctx, tree, Dm, J=J, Ej=Ej)
    jev = []
    for k in range(max(3, args.steps)):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        occk.farfield_J(ctx, tree, Dm, J=J, Ej=Ej)
        b.record(stream)
        jev.append((a, b))
    torch.cuda.synchronize()
    result["coulomb_j"] = {"ms": round(sum(a.elapsed_time(b) for a, b in jev) / len(jev), 4),
                           "E_J": float(Ej.item()), "lmax": L, "dtype": "f64",
                           "what": "far-field J^ff and E_J on the same tree, D = 2 C C^T"}
    # ---- occupied-pair screening: the same chain and tree with localised
    # occupied orbitals, unscreened and screened, in the main precision
    if args.screen_tau > 0 and args.workload == "chain":
        sl = inputs.alkane_localised(args.ncarbon, lmax=L)
        Cl = occk.fortran(torch.tensor(sl.C, dtype=torch.float64, device=dev))

        def timed_loc(tau, prec):
            ctx.set_pair_screen(tau)
            try:
                for _ in range(3):
                    occk.farfield_K(ctx, tree, Cl, prec=prec, K=K, Ex=Ex)
                ev = []
                nst = max(3, args.steps)
                st = {k: 0.0 for k in occk.STAGES}
                ctx.set_timing(True)
                for k in range(nst):
                    flush.fill_(float(k))
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    occk.farfield_K(ctx, tree, Cl, prec=prec, K=K, Ex=Ex)
                    b.record(stream)
                    ev.append((a, b))
                    for n_, v_ in ctx.timings().items():
                        st[n_] += v_ / nst
                ctx.set_timing(False)
                torch.cuda.synchronize()
                kept = ctx.pair_screen_count()
            finally:
                ctx.set_pair_screen(0.0)
            return (sum(a.elapsed_time(b) for a, b in ev) / len(ev), float(Ex.item()), K.clone(), kept,
                    {k: round(v, 4) for k, v in st.items()})

        ms0, E0, K0, _, st0 = timed_loc(0.0, args.prec)
        ms1, E1, K1, kept, st1 = timed_loc(args.screen_tau, args.prec)
        npair = system.nocc * (system.nocc + 1) // 2
        result["pair_screen"] = {
            "workload": sl.name + " (same geometry, basis and tree; localised occupied orbitals)",
            "tau": args.screen_tau, "kept_pairs": kept, "pairs": npair,
            "kept_fraction": round(kept / npair, 4),
            "ms_unscreened": round(ms0, 4), "ms_screened": round(ms1, 4),
            "speedup": round(ms0 / ms1, 3),
            "stage_ms_unscreened": st0, "stage_ms_screened": st1,
            "abs_dE_Eh": abs(E1 - E0),
            "rel_dK": float((K1 - K0).abs().max().item()) / float(K0.abs().max().item()),
            "dtype": "f64" if args.prec == "fp64" else args.prec}
        # the split-FP16 tensor-core form on the same localised orbitals,
        # against the FP64 unscreened energy
        if args.prec != "fp16x3":
            E64l = timed_loc(0.0, "fp64")[1]
            hs0, hE0, _, _, _ = timed_loc(0.0, "fp16x3")
            hs1, hE1, _, hkept, hst1 = timed_loc(args.screen_tau, "fp16x3")
            result["pair_screen"]["fp16x3"] = {
                "ms_unscreened": round(hs0, 4), "ms_screened": round(hs1, 4), "speedup": round(hs0 / hs1, 3),
                "kept_pairs": hkept, "stage_ms_screened": hst1,
                "abs_dE_vs_fp64_unscreened_Eh": abs(hE1 - E64l),
                "abs_dE_unscreened_vs_fp64_Eh": abs(hE0 - E64l)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(system, L, args.cpu_cols)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
