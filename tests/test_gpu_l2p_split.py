"""Step (e) with its K range split over several blocks (Eq. kri summed in
pieces, each into its own copy of the per-leaf K rows), in FP64, FP32 and on
the tensor core: any split count matches the unsplit FP64 path to the form's
accuracy (FP64: 1e-12, summation order only)."""
import numpy as np
import pytest

from paper_1708_05353_gb300 import inputs
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-4), ("fp16x3", 1e-5)])
@pytest.mark.parametrize("nsplit", [1, 2, 3, 8])
def test_l2p_split_matches(nsplit, prec, tol):
    from paper_1708_05353_gb300 import occk
    ctx = occk.Context(0)
    s = inputs.alkane(20, lmax=4, seed_k=4)
    tree = occk.Tree(ctx, s.basis, depth=s.depth, target_atoms_per_leaf=s.target_atoms_per_leaf)
    tree.pair_multipoles(4)
    C = torch.tensor(s.C, dtype=torch.float64, device="cuda:0")
    ctx.set_l2p_split(1)
    K64, E64 = occk.farfield_K(ctx, tree, C, prec="fp64", want_energy_host=True)
    ctx.set_l2p_split(nsplit)
    K, E = occk.farfield_K(ctx, tree, C, prec=prec, want_energy_host=True)
    ctx.set_l2p_split(0)
    assert rel_err(K.cpu().numpy(), K64.cpu().numpy()) < tol
    assert abs(E - E64) <= tol * abs(E64)
