"""GPU parity of occupied-pair screening (the paper's proposed extension to
localised orbitals, Sec. IV) through the C ABI against the oracle with the
same threshold: FP64 K and E within 1e-10 relative, the number of kept pairs
equal (an integer decision; thresholds sit in a gap of the pair-norm
distribution, 1e-6 relative wide in FP64 and 1e-4 in FP32, so both sides
decide every pair the same way), FP32 within 1e-4, FP16X3 (whose translations
then run on the SIMT kernel) within 1e-4.  A threshold of zero, or below every norm, is the unscreened method bit
for bit; a threshold above every norm leaves no far field."""
import numpy as np
import pytest

from oracle import fmm
from oracle import tree as otree
from paper_1708_05353_gb300 import inputs
from tests.helpers import rel_err, tau_in_gap

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_1708_05353_gb300 import occk
    c = occk.Context(0)
    yield c
    c.set_pair_screen(0.0)


def _gpu(ctx, s, L, prec="fp64", tau=0.0, tree=None):
    from paper_1708_05353_gb300 import occk
    if tree is None:
        tree = occk.Tree(ctx, s.basis, depth=s.depth, target_atoms_per_leaf=s.target_atoms_per_leaf)
        tree.pair_multipoles(L)
    C = torch.tensor(s.C, dtype=torch.float64, device="cuda:0")
    ctx.set_pair_screen(tau)
    try:
        K, E = occk.farfield_K(ctx, tree, C, prec=prec, want_energy_host=True)
        kept = ctx.pair_screen_count()
    finally:
        ctx.set_pair_screen(0.0)
    torch.cuda.synchronize()
    return tree, K.cpu().numpy(), E, kept


@pytest.fixture(scope="module")
def loc():
    s = inputs.small_sp_localised()
    tr = otree.build_tree(s.basis, s.depth, s.target_atoms_per_leaf)
    _, _, p = fmm.farfield(s, L=3, tree=tr, pair_tau=1.0, return_parts=True)
    return s, tr, p["norm2"]


@pytest.mark.parametrize("q", [0.2, 0.5, 0.8])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_screen_matches_oracle(ctx, loc, q, prec):
    s, tr, norm2 = loc
    # FP32 storage: the norms carry single-precision rounding of the
    # multipoles, so the threshold keeps a wider distance from every pair
    tau = tau_in_gap(norm2, q, gap=1e-6 if prec == "fp64" else 1e-4)
    Kr, Er, p = fmm.farfield(s, L=3, tree=tr, pair_tau=tau, return_parts=True)
    _, K, E, kept = _gpu(ctx, s, 3, prec=prec, tau=tau)
    assert kept == int(np.triu(p["keep"]).sum())
    bound = 1e-10 if prec == "fp64" else 1e-4
    assert rel_err(K, Kr) < bound
    assert abs(E - Er) <= bound * abs(Er)


def test_screen_below_every_norm_is_unscreened(ctx, loc):
    s, tr, norm2 = loc
    tree, K0, E0, kept0 = _gpu(ctx, s, 3)
    assert kept0 == -1
    _, K, E, kept = _gpu(ctx, s, 3, tau=1e-300, tree=tree)
    assert kept == s.nocc * (s.nocc + 1) // 2
    assert np.array_equal(K, K0) and E == E0


def test_screen_above_every_norm_leaves_nothing(ctx, loc):
    s, tr, norm2 = loc
    _, K, E, kept = _gpu(ctx, s, 3, tau=2.0 * float(np.sqrt(norm2.max())))
    assert kept == 0
    assert np.all(K == 0) and E == 0.0


def test_screen_chain_columns(ctx):
    """Localised orbitals on a 30-carbon chain (121 occupied, depth 4):
    several pair blocks of the tree passes, checked on three K columns."""
    from paper_1708_05353_gb300 import occk
    s = inputs.alkane_localised(30)
    tree = occk.Tree(ctx, s.basis, depth=s.depth, target_atoms_per_leaf=s.target_atoms_per_leaf)
    tree.pair_multipoles(2)
    tr = otree.build_tree(s.basis, s.depth, s.target_atoms_per_leaf)
    assert tr["depth"] == tree.info()["depth"] >= 3
    I = [0, 60, 120]
    _, _, p = fmm.farfield(s, L=2, tree=tr, pair_tau=1.0, i_subset=I, return_parts=True)
    tau = tau_in_gap(p["norm2"], 0.5)
    Kr, _ = fmm.farfield(s, L=2, tree=tr, pair_tau=tau, i_subset=I)
    _, K, E, kept = _gpu(ctx, s, 2, tau=tau, tree=tree)
    assert 0 < kept < s.nocc * (s.nocc + 1) // 2
    assert rel_err(K[:, I], Kr) < 1e-10


@pytest.mark.parametrize("q", [0.3, 0.7])
def test_screen_fp16x3(ctx, loc, q):
    """The split-FP16 tensor-core form screens too (its tree passes then run on
    the SIMT kernel): its norms carry the form's ~1e-6 relative error, so the
    threshold keeps 1e-3 away from every pair; K and E follow the screened
    oracle within the form's bounds."""
    s, tr, norm2 = loc
    tau = tau_in_gap(norm2, q, gap=1e-3)
    Kr, Er, p = fmm.farfield(s, L=3, tree=tr, pair_tau=tau, return_parts=True)
    _, K, E, kept = _gpu(ctx, s, 3, prec="fp16x3", tau=tau)
    assert kept == int(np.triu(p["keep"]).sum())
    assert rel_err(K, Kr) < 1e-4
    assert abs(E - Er) <= 1e-5 * abs(Er)
