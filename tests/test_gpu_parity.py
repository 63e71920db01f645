"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances: FP64 path max|dK|/max|K| <= 1e-10 and |dE|/|E| <= 1e-10 (the
plain-FP64 bar); FP32 path 1e-4 relative in K (single-precision contractions
over a few hundred terms, relative unit round-off 6e-8 times condition
growth), stated per test.
"""
import numpy as np
import pytest

from oracle import fmm, solid
from oracle import tree as otree
from paper_1708_05353_gb300 import inputs
from tests.helpers import complex_to_real, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_1708_05353_gb300 import occk
    return occk.Context(0)


def _run(ctx, s, L, prec="fp64", depth=None, ranks=None):
    from paper_1708_05353_gb300 import occk
    d = s.depth if depth is None else depth
    tree = occk.Tree(ctx, s.basis, depth=d, target_atoms_per_leaf=s.target_atoms_per_leaf)
    tree.pair_multipoles(L)
    policy = 0
    if ranks is not None:
        tree.set_edge_lmax(ranks)
        policy = 1
    C = torch.tensor(s.C, dtype=torch.float64, device="cuda:0")
    K, E = occk.farfield_K(ctx, tree, C, prec=prec, lmax_policy=policy, want_energy_host=True)
    torch.cuda.synchronize()
    return tree, K.cpu().numpy(), E


def _oracle(s, L, depth=None, i_subset=None, lmax_edges=None, parts=False):
    d = s.depth if depth is None else depth
    tr = otree.build_tree(s.basis, d, s.target_atoms_per_leaf)
    out = fmm.farfield(s, L=L, tree=tr, i_subset=i_subset, lmax_edges=lmax_edges,
                       return_parts=parts)
    return tr, out


def test_pair_multipoles_match(ctx):
    from paper_1708_05353_gb300 import occk
    s = inputs.small_sp(natom=5, nocc=3, spacing=3.0, depth=3)
    L = 6
    tree = occk.Tree(ctx, s.basis, depth=3)
    tree.pair_multipoles(L)
    got = occk.debug_fetch_pair_mult(ctx, tree, s.basis.shell_l, stream=0)
    tr = otree.build_tree(s.basis, 3, 8.0)
    Op = fmm.pair_multipoles(s.basis, tr, L)
    ref = np.concatenate([complex_to_real(o, L).reshape(-1, (L + 1) ** 2) for o in Op], axis=0)
    assert got.shape == ref.shape
    assert rel_err(got, ref) < 1e-12


@pytest.mark.parametrize("L", [0, 2, 3, 6])
def test_fp64_small_sp(ctx, L):
    s = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    tree, K, E = _run(ctx, s, L)
    _, (Kr, Er) = _oracle(s, L)
    assert rel_err(K, Kr) < 1e-10
    assert abs(E - Er) <= 1e-10 * abs(Er)


def test_fp64_intermediates(ctx):
    """Occupied multipoles and local expansions of every box, step by step."""
    from paper_1708_05353_gb300 import occk
    s = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    L = 3
    tree, K, E = _run(ctx, s, L)
    tr, (Kr, Er, parts) = _oracle(s, L, parts=True)
    Ob = occk.debug_fetch(ctx, tree, "obox", nocc=s.nocc, stream=0)
    Mb = occk.debug_fetch(ctx, tree, "mbox", nocc=s.nocc, stream=0)
    n = s.nocc
    Or = complex_to_real(np.moveaxis(parts["Obox"], 1, -1), L)       # [box, i, j, nc]
    Mr = complex_to_real(np.moveaxis(parts["Mbox"], 1, -1), L)
    first = tr["level_off"][2]
    Og = np.moveaxis(Ob.reshape(Ob.shape[0], -1, n, n), 1, -1)
    Mg = np.moveaxis(Mb.reshape(Mb.shape[0], -1, n, n), 1, -1)
    assert rel_err(Og[first:], Or[first:]) < 1e-12
    assert rel_err(Mg[first:], Mr[first:]) < 1e-11


def test_fp64_line40(ctx):
    s = inputs.tiny_line()
    tree, K, E = _run(ctx, s, 2)
    _, (Kr, Er) = _oracle(s, 2)
    assert rel_err(K, Kr) < 1e-10
    assert abs(E - Er) <= 1e-10 * abs(Er)


def test_fp64_water_3d(ctx):
    """3-D cluster with s and p shells, ragged pair tiles (nocc = 60)."""
    s = inputs.water(nmol=12, lmax=4)
    tree, K, E = _run(ctx, s, 4, depth=2)
    _, (Kr, Er) = _oracle(s, 4, depth=2)
    assert rel_err(K, Kr) < 1e-10
    assert abs(E - Er) <= 1e-10 * abs(Er)


def test_fp32_water_3d(ctx):
    s = inputs.water(nmol=12, lmax=4)
    tree, K, E = _run(ctx, s, 4, prec="fp32", depth=2)
    _, (Kr, Er) = _oracle(s, 4, depth=2)
    assert rel_err(K, Kr) < 1e-4
    assert abs(E - Er) <= 1e-5 * abs(Er)


def test_fp64_chain_columns(ctx):
    """60-carbon chain, nocc = 241 (several 64-wide tiles and a ragged tail)."""
    s = inputs.alkane(60, lmax=2)
    tree, K, E = _run(ctx, s, 2)
    I = [0, 77, 240]
    _, (Kr, Er) = _oracle(s, 2, i_subset=I)
    assert rel_err(K[:, I], Kr) < 1e-10


def test_edge_case_no_far_field(ctx):
    """Depth 1: every box neighbours every other, K^ff = 0 and E^ff = 0."""
    s = inputs.small_sp(natom=4, nocc=2, spacing=3.0, depth=1)
    tree, K, E = _run(ctx, s, 2, depth=1)
    assert np.all(K == 0) and E == 0.0


def test_edge_case_single_orbital(ctx):
    s = inputs.small_sp(natom=6, nocc=1, spacing=3.0, depth=3)
    tree, K, E = _run(ctx, s, 3)
    _, (Kr, Er) = _oracle(s, 3)
    assert rel_err(K, Kr) < 1e-10


def test_per_edge_lmax(ctx):
    s = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    L = 4
    tr = otree.build_tree(s.basis, 3, 8.0)
    rng = np.random.default_rng(3)
    ranks = rng.integers(0, L + 1, size=len(tr["m2l_tgt"]))
    tree, K, E = _run(ctx, s, L, ranks=ranks)
    _, (Kr, Er) = _oracle(s, L, lmax_edges=ranks)
    assert rel_err(K, Kr) < 1e-10
    assert abs(E - Er) <= 1e-10 * abs(Er)


def test_repeat_is_deterministic(ctx):
    s = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    _, K1, E1 = _run(ctx, s, 3)
    _, K2, E2 = _run(ctx, s, 3)
    assert np.array_equal(K1, K2) and E1 == E2
