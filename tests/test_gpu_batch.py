"""Batched far field: uneven systems, in either batch mode (one persistent,
level-synchronous launch sequence over all systems, or every system's own
pipeline on forked streams), graph-captured, must reproduce each system's
single-system result (FP64: 1e-12 relative; FP32: 1e-5), include a system
with no far field (depth 1), replay from the CUDA graph bit-identically, match
the FP64 oracle, and the autotuner must write and reuse its cache."""
import os

import numpy as np
import pytest

from oracle import fmm
from oracle import tree as otree
from paper_1708_05353_gb300 import inputs
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _systems(L=4):
    a = inputs.alkane(20, lmax=L, seed_k=4)
    w = inputs.water(12, lmax=L, seed_k=4, geom_seed=4100)
    w.depth = 2
    w1 = inputs.water(8, lmax=L, seed_k=4, geom_seed=4200)
    w1.depth = 1
    sp = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3, lmax=L)
    return [a, w, w1, sp]


def _batch(ctx, systems, prec, L=4):
    from paper_1708_05353_gb300 import occk
    trees = []
    for s in systems:
        t = occk.Tree(ctx, s.basis, depth=s.depth, target_atoms_per_leaf=s.target_atoms_per_leaf)
        t.pair_multipoles(L)
        trees.append(t)
    b = occk.Batch(ctx, trees, [s.nocc for s in systems], prec=prec)
    for k, s in enumerate(systems):
        c, _, _, ld = b.buffers(k)
        C = occk.device_view(c, (s.nocc, ld), torch.float64, "cuda:0")
        C.copy_(torch.tensor(s.C.T, dtype=torch.float64))
    return trees, b


def _read(b, systems):
    from paper_1708_05353_gb300 import occk
    out = []
    for k, s in enumerate(systems):
        _, kp, ep, ld = b.buffers(k)
        K = occk.device_view(kp, (s.nocc, ld), torch.float64, "cuda:0").t().cpu().numpy()
        E = occk.device_view(ep, (len(systems),), torch.float64, "cuda:0")[k].item()
        out.append((K, E))
    return out


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_batch_matches_single(prec, tol, mode):
    """Both batch modes: level-synchronous persistent kernels (0) and every
    system's own pipeline on forked streams (1)."""
    from paper_1708_05353_gb300 import occk
    ctx = occk.Context(0)
    systems = _systems()
    trees, b = _batch(ctx, systems, prec)
    b.set_config(tile=64 if prec == "fp64" else 128, mode=mode)
    b.run(use_graph=False)
    torch.cuda.synchronize()
    got = _read(b, systems)
    for s, t, (K, E) in zip(systems, trees, got):
        C = torch.tensor(s.C, dtype=torch.float64, device="cuda:0")
        Ks, Es = occk.farfield_K(ctx, t, C, prec=prec, want_energy_host=True)
        Ks = Ks.cpu().numpy()
        if t.info()["depth"] < 2:
            assert np.all(K == 0) and E == 0.0
            continue
        assert rel_err(K, Ks) < tol
        assert abs(E - Es) <= tol * abs(Es)


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_graph_replay_and_oracle(mode):
    from paper_1708_05353_gb300 import occk
    ctx = occk.Context(0)
    systems = _systems()
    trees, b = _batch(ctx, systems, "fp64")
    b.set_config(tile=64, mode=mode)
    b.run(use_graph=False)
    torch.cuda.synchronize()
    ref = _read(b, systems)
    for _ in range(2):
        b.run(use_graph=True)
        torch.cuda.synchronize()
        got = _read(b, systems)
        for (K1, E1), (K2, E2) in zip(ref, got):
            assert np.array_equal(K1, K2) and E1 == E2
    s = systems[1]
    Kr, Er = fmm.farfield(s, L=4, tree=otree.build_tree(s.basis, s.depth, 8.0))
    assert rel_err(got[1][0], Kr) < 1e-10
    assert abs(got[1][1] - Er) <= 1e-10 * abs(Er)


def test_batch_autotune_cache(tmp_path):
    from paper_1708_05353_gb300 import occk
    ctx = occk.Context(0)
    systems = _systems()
    trees, b = _batch(ctx, systems, "fp32")
    path = str(tmp_path / "tune.txt")
    cfg = b.tune(path)
    assert os.path.exists(path)
    assert cfg["chunk"] in (4, 9, 16, 21, 25) and cfg["tile"] in (64, 128) and cfg["mode"] in (0, 1)
    line = open(path).read().split()
    assert [int(x) for x in line[1:5]] == [cfg["chunk"], cfg["blocks_per_sm"], cfg["tile"], cfg["mode"]]
    # cached: the same configuration without re-timing
    assert b.tune(path) == cfg
    b.run(use_graph=True)
    torch.cuda.synchronize()
    got = _read(b, systems)
    C = torch.tensor(systems[0].C, dtype=torch.float64, device="cuda:0")
    Ks, Es = occk.farfield_K(ctx, trees[0], C, prec="fp32", want_energy_host=True)
    assert rel_err(got[0][0], Ks.cpu().numpy()) < 1e-5
