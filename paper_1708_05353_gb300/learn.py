"""Training and evaluation of the learned per-edge M2L rank selector.

Labels come from the method's own truncation errors: a far-field run at the
reference rank L_ref = 10 leaves the occupied multipoles of every box on the
device; occk_edge_energies splits the far-field energy over M2L edges for
every truncation rank (exact, since M2M and L2L re-expand exactly), and the
label of an edge at rank L is log10 |e_edge(L) - e_edge(L_ref)|.  Features are
computed by occk_edge_features from the same multipoles.  Training and
inference run in the library's CUDA kernels (FP32 Adam, FP16 inference); this
module only moves arrays.

    python -m paper_1708_05353_gb300.learn train --out lmax_selector.npz
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import inputs, occk

LREF = 10
RANKS = list(range(2, 2 + occk.MLP_NOUT))     # 2..9
HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "lmax_selector.npz")


def _torch():
    import torch
    return torch


def run_far_field(ctx, system, L, prec="fp64", policy=0, depth=None, tree=None):
    torch = _torch()
    if tree is None:
        d = system.depth if depth is None else depth
        tree = occk.Tree(ctx, system.basis, depth=d, target_atoms_per_leaf=system.target_atoms_per_leaf)
        tree.pair_multipoles(L)
    C = occk.fortran(torch.tensor(system.C, dtype=torch.float64, device=f"cuda:{ctx.device}"))
    K, E = occk.farfield_K(ctx, tree, C, prec=prec, lmax_policy=policy, want_energy_host=True)
    return tree, K, E


def edge_dataset(ctx, system, Lref=LREF, prec="fp64", depth=None):
    """Features [n_edge, 16] and labels [n_edge, 8] (log10 Eh) of one system."""
    tree, K, E = run_far_field(ctx, system, Lref, prec=prec, depth=depth)
    F = occk.edge_features(ctx, tree).cpu().numpy().astype(np.float64)
    Ee = occk.edge_energies(ctx, tree).cpu().numpy()
    ref = Ee[:, Lref:Lref + 1]
    err = np.abs(Ee[:, RANKS] - ref)
    floor = 1e-15 * np.abs(ref) + 1e-20
    Y = np.log10(err + floor)
    return F, Y, dict(E=E, edge_energy=Ee, nedge=F.shape[0], tree=tree.info())


def train(ctx, X, Y, steps=4000, lr=2e-3, seed=1, quantile=0.9):
    """Standardise, initialise and train on the device; then calibrate: the
    predicted log10 errors are shifted up by the `quantile` of the training
    residuals of each output, so that the rank choice errs on the safe side.
    Returns (final loss, per-output shift)."""
    torch = _torch()
    mx, sx = X.mean(axis=0), X.std(axis=0) + 1e-3
    my, sy = Y.mean(axis=0), Y.std(axis=0) + 1e-3
    norm = np.concatenate([mx, sx, my, sy]).astype(np.float32)
    occk.mlp_init(ctx, seed)
    p, _ = occk.mlp_get(ctx)
    occk.mlp_set(ctx, p, norm)
    dev = f"cuda:{ctx.device}"
    Xd = torch.tensor(X, dtype=torch.float32, device=dev).contiguous()
    Td = torch.tensor((Y - my) / sy, dtype=torch.float32, device=dev).contiguous()
    loss = occk.mlp_train(ctx, Xd, Td, steps, lr)
    pred = occk.mlp_predict(ctx, Xd).cpu().numpy().astype(np.float64)
    shift = np.maximum(np.quantile(Y - pred, quantile, axis=0), 0.0)
    p, norm = occk.mlp_get(ctx)
    norm[2 * occk.MLP_NIN:2 * occk.MLP_NIN + occk.MLP_NOUT] += shift.astype(np.float32)
    occk.mlp_set(ctx, p, norm)
    return loss, shift


def lagrangian_choice(log_err, Lmax, tau):
    """The device's rank rule, on the host: minimise sum (L+1)^4 subject to
    sum err <= tau by bisection on log10 of the multiplier."""
    ranks = np.arange(2, Lmax + 1)
    err = np.zeros((log_err.shape[0], len(ranks)))
    for k, L in enumerate(ranks):
        err[:, k] = 10.0 ** log_err[:, L - 2] if L - 2 < log_err.shape[1] else 0.0
    cost = (ranks + 1.0) ** 4

    def pick(loglam):
        v = cost[None, :] + 10.0 ** loglam * err
        j = np.argmin(v, axis=1)
        return ranks[j], err[np.arange(len(j)), j].sum()
    lo, hi = -10.0, 60.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if pick(mid)[1] <= tau:
            hi = mid
        else:
            lo = mid
    return pick(hi)[0]


def save(ctx, path):
    p, n = occk.mlp_get(ctx)
    np.savez(path, params=p, norm=n, nin=occk.MLP_NIN, hidden=occk.MLP_HIDDEN, nout=occk.MLP_NOUT,
             ranks=np.array(RANKS), lref=LREF)


def load(ctx, path=DEFAULT_WEIGHTS):
    z = np.load(path)
    occk.mlp_set(ctx, z["params"], z["norm"])


def m2l_cost(ranks):
    return float(np.sum((np.asarray(ranks, dtype=np.float64) + 1.0) ** 4))


def _timed(fn):
    torch = _torch()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def compare(ctx, system, tau, Lref=LREF, prec="fp64", depth=None, fixed=(2, 3, 4, 5, 6, 7, 8, 9, 10)):
    """Learned ranks vs fixed ranks on one system.  Errors are measured against
    the rank-Lref energy; the M2L cost is sum over edges of (L_e+1)^4."""
    (tree, K, Eref), t_ref = _timed(lambda: run_far_field(ctx, system, Lref, prec=prec, depth=depth))
    # a second run of the same tree for the far-field time without set-up
    _, t_ref = _timed(lambda: run_far_field(ctx, system, Lref, prec=prec, tree=tree))
    nedge = tree.info()["nm2l"]
    Ee = occk.edge_energies(ctx, tree).cpu().numpy()
    rows = {}
    for L in fixed:
        E_L = float(np.sum(Ee[:, L])) if nedge else 0.0
        rows[L] = dict(err=abs(E_L - Eref), cost=m2l_cost([L] * nedge))
    occk.set_learned_tau(ctx, tau)
    (_, K2, E_learn), t_learn = _timed(lambda: run_far_field(ctx, system, Lref, prec=prec, policy=2, tree=tree))
    ranks = occk.edge_ranks(ctx, tree)
    learned = dict(err=abs(E_learn - Eref), cost=m2l_cost(ranks), ranks_hist=np.bincount(ranks, minlength=Lref + 1).tolist())
    # cheapest fixed rank at least as accurate as the learned choice
    ok = [L for L in fixed if rows[L]["err"] <= max(learned["err"], 1e-300)]
    matched = min(ok) if ok else Lref
    # best possible choice: the same rule on the true edge errors
    optimal = None
    if nedge:
        true_log = np.log10(np.abs(Ee[:, RANKS] - Ee[:, Lref:Lref + 1]) + 1e-300)
        r_opt = lagrangian_choice(true_log, Lref, tau)
        E_opt = float(np.sum(Ee[np.arange(nedge), r_opt]))
        optimal = dict(err=abs(E_opt - Eref), cost=m2l_cost(r_opt))
    learned["time_s"] = t_learn
    return dict(E_ref=Eref, tau=tau, fixed=rows, learned=learned, optimal=optimal, matched_fixed_rank=matched,
                time_fixed_lref_s=t_ref, speedup_time_vs_lref=t_ref / max(t_learn, 1e-9),
                gain_vs_matched=rows[matched]["cost"] / max(learned["cost"], 1.0),
                gain_vs_lref=rows[Lref]["cost"] / max(learned["cost"], 1.0), nedge=nedge)


def training_systems(scale="full"):
    """Workloads of the training set: the chain, water-cluster and batched
    shapes (configs 2-4 of this project's workload list); `small` gives
    reduced sizes for tests."""
    if scale == "small":
        chains = [inputs.alkane(n, lmax=LREF, seed_k=k) for n, k in ((30, 2), (36, 7), (44, 8))]
        waters = [inputs.water(n, lmax=LREF, seed_k=k, geom_seed=g)
                  for n, k, g in ((20, 3, 3000), (27, 4, 4321), (24, 9, 9000))]
        for s in waters:
            s.depth = 2      # small clusters: two subdivisions so that M2L edges exist
        return chains + waters
    out = [inputs.alkane(150, lmax=LREF), inputs.water(100, lmax=LREF), inputs.flake(lmax=LREF)]
    out += [inputs.alkane(n, lmax=LREF, seed_k=4) for n in (50, 100)]
    out += [inputs.water(n, lmax=LREF, seed_k=4, geom_seed=4000 + 10 * k)
            for k, n in enumerate((20, 30, 40, 50, 60))]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "eval"])
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--scale", default="full")
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--tau", type=float, default=1e-6)
    args = ap.parse_args()
    ctx = occk.Context(0)
    if args.cmd == "train":
        Xs, Ys, meta = [], [], []
        t0 = time.time()
        for s in training_systems(args.scale):
            X, Y, m = edge_dataset(ctx, s)
            Xs.append(X)
            Ys.append(Y)
            meta.append(dict(name=s.name, nedge=m["nedge"], E=m["E"]))
            print(json.dumps(meta[-1]), flush=True)
        X = np.concatenate(Xs)
        Y = np.concatenate(Ys)
        t1 = time.time()
        loss, shift = train(ctx, X, Y, steps=args.steps, lr=args.lr)
        t2 = time.time()
        save(ctx, args.out)
        print(json.dumps(dict(samples=int(X.shape[0]), loss=loss, shift=shift.tolist(), label_s=t1 - t0,
                              train_s=t2 - t1, out=args.out)), flush=True)
    else:
        load(ctx, args.out)
        s = inputs.protein_like(lmax=LREF)
        res = compare(ctx, s, args.tau)
        res["system"] = s.name
        res["nao"] = s.basis.nao
        res["nocc"] = s.nocc
        print(json.dumps(res, default=float), flush=True)


if __name__ == "__main__":
    main()
