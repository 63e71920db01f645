"""FP32 steps (a) and (e) from 4 integer slices on the tensor core
(occk_set_fp32_slices).

The FP32 form's two GEMM-shaped steps, the full transform (Eq. motrans) and
the K assembly (Eq. kri), run on the engine of the sliced FP64 form with 4
slices of at most 7 bits per operand: every FP32 operand lies within 2^-28 of
its row's largest entry in the slices, the products are summed exactly and
combined in FP64, so neither step adds FP32 rounding nor the tensor core's
accumulation bias.  The half transform and the tree passes stay FP32 SIMT.
K follows the oracle's exact columns (tests/golden/oracle_columns.npz) at the
FP32 bar (1e-4 relative) and E within 1e-6 Eh; the tests also print the plain
FP32 form's error on the same build.
"""
import os

import numpy as np
import pytest

from paper_1708_05353_gb300 import inputs
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLD = np.load(os.path.join(os.path.dirname(__file__), "golden", "oracle_columns.npz"))
SYSTEMS = {
    "chain60": lambda: inputs.alkane(60, lmax=2),
    "protein": lambda: inputs.protein_like(lmax=2),
}


@pytest.fixture(scope="module")
def ctx():
    from paper_1708_05353_gb300 import occk
    c = occk.Context(0)
    yield c
    c.set_fp32_slices(0)


def _run(ctx, tree, C, slices, prec="fp32"):
    from paper_1708_05353_gb300 import occk
    ctx.set_fp32_slices(slices)
    try:
        K, E = occk.farfield_K(ctx, tree, C, prec=prec, want_energy_host=True)
        occk.device_status(ctx)
    finally:
        ctx.set_fp32_slices(0)
    return K.clone(), E


@pytest.mark.parametrize("name,L", [("chain60", 2), ("chain60", 6), ("protein", 2)])
def test_fp32_sliced_oracle_columns(ctx, name, L):
    from paper_1708_05353_gb300 import occk
    s = SYSTEMS[name]()
    tree = occk.Tree(ctx, s.basis, depth=s.depth, target_atoms_per_leaf=s.target_atoms_per_leaf)
    tree.pair_multipoles(L)
    C = torch.tensor(s.C, dtype=torch.float64, device="cuda:0")
    cols = GOLD[f"{name}/cols"]
    Kr = GOLD[f"{name}/L{L}/K"]
    Er = float(GOLD[f"{name}/L{L}/E_cols"])
    K, E = _run(ctx, tree, C, 4)
    K0, E0 = _run(ctx, tree, C, 0)
    K64, E64 = _run(ctx, tree, C, 0, prec="fp64")
    idx = torch.as_tensor(cols, device=K.device)
    err = rel_err(K[:, idx].cpu().numpy(), Kr)
    err0 = rel_err(K0[:, idx].cpu().numpy(), Kr)
    Ec = -0.5 * float(np.sum(s.C[:, cols] * K[:, idx].cpu().numpy()))
    print(f"{name} L={L}: sliced FP32 max|dK|/max|K| {err:.2e} (SIMT FP32 {err0:.2e}), "
          f"|dE| vs FP64 {abs(E - E64):.2e} (SIMT FP32 {abs(E0 - E64):.2e})")
    assert err < 1e-4
    assert abs(Ec - Er) <= 1e-4 * abs(Er)
    assert abs(E - E64) < 1e-6


def test_fp32_slices_argument(ctx):
    from paper_1708_05353_gb300 import occk
    for bad in (-1, 1, 6, 7):
        with pytest.raises(occk.OcckError):
            ctx.set_fp32_slices(bad)
