"""The sibling-grouped FP32 M2L (+ L2L) against the per-target pass.

Both compute, for every target box, the sum over its interaction list of
T(target, source) O(source) in ascending source order, then the parent's
local expansion translated down (Eqs. fmmex, fmm2, fmm3), so the two kernels
must give bit-identical K in every precision whose translations run on the
FP32 SIMT path (FP32, and the tensor-core forms at low rank), with and without
occupied-pair screening; the grouped result also follows the oracle's exact
columns (tests/golden/oracle_columns.npz) within the FP32 bound.
"""
import os

import numpy as np
import pytest

from paper_1708_05353_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLD = np.load(os.path.join(os.path.dirname(__file__), "golden", "oracle_columns.npz"))


@pytest.fixture(scope="module")
def ctx():
    from paper_1708_05353_gb300 import occk
    c = occk.Context(0)
    yield c
    c.set_m2l_group(-1)
    c.set_pair_screen(0.0)


def _run(ctx, tree, C, prec, mode, tau=0.0):
    from paper_1708_05353_gb300 import occk
    ctx.set_m2l_group(mode)
    ctx.set_pair_screen(tau)
    try:
        K, E = occk.farfield_K(ctx, tree, C, prec=prec, want_energy_host=True)
    finally:
        ctx.set_m2l_group(-1)
        ctx.set_pair_screen(0.0)
    return K.clone(), E


def _setup(ctx, s, L, depth=None):
    from paper_1708_05353_gb300 import occk
    tree = occk.Tree(ctx, s.basis, depth=s.depth if depth is None else depth,
                     target_atoms_per_leaf=s.target_atoms_per_leaf)
    tree.pair_multipoles(L)
    return tree, occk.fortran(torch.tensor(s.C, dtype=torch.float64, device="cuda:0"))


@pytest.mark.parametrize("name,L", [("water12", 2), ("water12", 3), ("water12", 1), ("chain60", 2)])
@pytest.mark.parametrize("prec", ["fp32", "fp16x3", "tf32"])
def test_grouped_equals_per_target(ctx, name, L, prec):
    s = inputs.water(nmol=12, lmax=L) if name == "water12" else inputs.alkane(60, lmax=L)
    tree, C = _setup(ctx, s, L, depth=2 if name == "water12" else None)
    K0, E0 = _run(ctx, tree, C, prec, 0)
    K1, E1 = _run(ctx, tree, C, prec, 1)
    assert torch.equal(K0, K1) and E0 == E1


def test_grouped_protein_levels_and_oracle(ctx):
    """The protein-sized cluster (two M2L levels, L2L into level 3): grouped
    and per-target bit for bit, and both at the FP32 bound of the oracle's
    columns."""
    s = inputs.protein_like(lmax=2)
    tree, C = _setup(ctx, s, 2)
    assert tree.info()["depth"] == 3
    K0, _ = _run(ctx, tree, C, "fp32", 0)
    K1, _ = _run(ctx, tree, C, "fp32", 1)
    assert torch.equal(K0, K1)
    cols = GOLD["protein/cols"]
    Kr = GOLD["protein/L2/K"]
    Kc = K1[:, torch.as_tensor(cols, device=K1.device)].cpu().numpy()
    assert float(np.max(np.abs(Kc - Kr)) / np.max(np.abs(Kr))) < 1e-4


def test_grouped_screened(ctx):
    """With occupied-pair screening the tree passes run on compacted kept
    pairs (a device-side live count); grouped and per-target agree bit for bit."""
    s = inputs.alkane_localised(30)
    tree, C = _setup(ctx, s, 2)
    K0, E0 = _run(ctx, tree, C, "fp32", 0, tau=1e-4)
    K1, E1 = _run(ctx, tree, C, "fp32", 1, tau=1e-4)
    assert torch.equal(K0, K1) and E0 == E1


def test_mode_argument(ctx):
    from paper_1708_05353_gb300 import occk
    with pytest.raises(occk.OcckError):
        ctx.set_m2l_group(2)
