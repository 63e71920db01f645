"""Stored expected values (tests/golden/line40_farfield.json, written by
tests/golden/make_golden.py from the FP64 oracle only) for the 40-atom line
workload: the oracle must reproduce them, the ranks must approach the exact
far field from four-centre integrals, and the CUDA FP64 path must match them
at every rank 0..6 (1e-10 relative, the plain-FP64 bar)."""
import json
import os

import numpy as np
import pytest

from oracle import fmm
from oracle import tree as otree
from paper_1708_05353_gb300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "line40_farfield.json")))


def test_oracle_reproduces_golden():
    s = inputs.tiny_line()
    tr = otree.build_tree(s.basis, s.depth, s.target_atoms_per_leaf)
    for L in (0, 2):
        K, E = fmm.farfield(s, L=L, tree=tr)
        assert abs(E - GOLD["energy_by_rank"][str(L)]) <= 1e-12 * abs(E)
    K2, _ = fmm.farfield(s, L=2, tree=tr)
    assert np.allclose(K2[0], GOLD["K_row0_rank2"], rtol=1e-12, atol=1e-15)


def test_golden_ranks_approach_exact():
    Ex = GOLD["energy_exact"]
    err = {int(L): abs(E - Ex) for L, E in GOLD["energy_by_rank"].items()}
    assert err[6] < err[2] < err[1]
    assert err[6] < 2e-4 * abs(Ex)


@pytest.mark.gpu
def test_cuda_fp64_matches_golden():
    torch = pytest.importorskip("torch")
    from paper_1708_05353_gb300 import occk
    s = inputs.tiny_line()
    ctx = occk.Context(0)
    C = torch.tensor(s.C, dtype=torch.float64, device="cuda:0")
    for L in range(0, 7):
        tree = occk.Tree(ctx, s.basis, depth=s.depth, target_atoms_per_leaf=s.target_atoms_per_leaf)
        tree.pair_multipoles(L)
        K, E = occk.farfield_K(ctx, tree, C, prec="fp64", want_energy_host=True)
        Eg = GOLD["energy_by_rank"][str(L)]
        assert abs(E - Eg) <= 1e-10 * abs(Eg), (L, E, Eg)
        if L == 2:
            row = K.cpu().numpy()[0]
            ref = np.asarray(GOLD["K_row0_rank2"])
            assert np.max(np.abs(row - ref)) <= 1e-10 * np.max(np.abs(ref))
