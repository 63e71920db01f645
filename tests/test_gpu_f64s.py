"""FP64 steps (a) and (e) from integer slices on the tensor core
(occk_set_fp64_slices).

The full transform O^{ij}_lm = sum_r C_ri O^{rj}_lm (Eq. motrans) and the K
assembly K_ri = 2 sum_X sum_{j,lm} O^{rj,X}_lm Mcal^{ij}_lm(X) (Eq. kri) are
computed from the error-free splitting of their operands into 7-bit integer
slices (Ozaki, Ogita, Oishi and Rump 2012) with exact sums of the slice
products on FP16 tensor-core MMAs; every other step is the FP64 path.  The
result differs from the DFMA forms only by the slices' truncation, about
2^-49 (7 slices) or 2^-42 (6 slices) of the largest row and column entries
per product.  Against the oracle's exact columns
(tests/golden/oracle_columns.npz) that is about 1e-12 of max|K| for 7 slices,
inside the plain FP64 bar (1e-10); the tests hold it to 1e-11 (7 slices) and
1e-9 (6 slices), against the oracle and against the DFMA forms.  Cases:
several full 128-row and 32-orbital tiles (the 60-carbon chain, 241 orbitals,
at L = 2 and L = 6), the benchmark's protein-sized cluster, a long K range at
L = 10 (121 components, 23 exact chunks per step (e) tile) and a small system
whose step (e) tiles are split along K to fill the GPU.  From L = 4 on, M2L
(Eqs. fmmex, fmm2) runs from slices too, with the parent's L2L added in
double-FP32; it is compared with the double-FP32 M2L, with fixed and
per-edge ranks, and the batching of its pair tiles is bit-exact.
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
    "chain20": lambda: inputs.alkane(20, lmax=10, seed_k=4),
    "protein": lambda: inputs.protein_like(lmax=2),
}


@pytest.fixture(scope="module")
def ctx():
    from paper_1708_05353_gb300 import occk
    c = occk.Context(0)
    yield c
    c.set_fp64_slices(0)
    c.set_pair_screen(0.0)


def _build(ctx, s, L):
    from paper_1708_05353_gb300 import occk
    tree = occk.Tree(ctx, s.basis, depth=s.depth, target_atoms_per_leaf=s.target_atoms_per_leaf)
    tree.pair_multipoles(L)
    return tree, torch.tensor(s.C, dtype=torch.float64, device="cuda:0")


def _run(ctx, tree, C, slices, tau=0.0):
    from paper_1708_05353_gb300 import occk
    ctx.set_fp64_slices(slices)
    ctx.set_pair_screen(tau)
    try:
        K, E = occk.farfield_K(ctx, tree, C, prec="fp64", want_energy_host=True)
        occk.device_status(ctx)
    finally:
        ctx.set_fp64_slices(0)
        ctx.set_pair_screen(0.0)
    return K.clone(), E


@pytest.mark.parametrize("name,L,slices,bound", [("chain60", 2, 7, 1e-11), ("chain60", 6, 7, 1e-11),
                                                 ("chain60", 2, 6, 1e-9), ("chain20", 10, 7, 1e-11),
                                                 ("protein", 2, 7, 1e-11)])
def test_sliced_l2p_oracle_columns(ctx, name, L, slices, bound):
    s = SYSTEMS[name]()
    tree, C = _build(ctx, s, L)
    cols = GOLD[f"{name}/cols"]
    Kr = GOLD[f"{name}/L{L}/K"]
    Er = float(GOLD[f"{name}/L{L}/E_cols"])
    K, E = _run(ctx, tree, C, slices)
    K0, E0 = _run(ctx, tree, C, 0)
    Kc = K[:, torch.as_tensor(cols, device=K.device)].cpu().numpy()
    err = rel_err(Kc, Kr)
    Ec = -0.5 * float(np.sum(s.C[:, cols] * Kc))
    d_dfma = float((K - K0).abs().max() / K0.abs().max())
    print(f"{name} L={L} {slices} slices: max|dK|/max|K| vs oracle {err:.2e}, vs DFMA {d_dfma:.2e}, "
          f"|dE_cols| {abs(Ec - Er):.2e}, |E - E_dfma| {abs(E - E0):.2e}")
    assert err < bound
    assert abs(Ec - Er) <= bound * abs(Er)
    assert d_dfma < bound
    assert abs(E - E0) <= bound * abs(E0)


def test_sliced_l2p_split_small_system(ctx):
    """A water cluster has few tiles, so each is split along K (one K-row copy
    per split, summed by the reduction); the result follows the DFMA form."""
    s = inputs.water(nmol=12, lmax=4)
    from paper_1708_05353_gb300 import occk
    tree = occk.Tree(ctx, s.basis, depth=2)
    tree.pair_multipoles(4)
    C = torch.tensor(s.C, dtype=torch.float64, device="cuda:0")
    K, E = _run(ctx, tree, C, 7)
    K0, E0 = _run(ctx, tree, C, 0)
    d = float((K - K0).abs().max() / K0.abs().max())
    print(f"water12 L=4: vs DFMA {d:.2e}, |dE| {abs(E - E0):.2e}")
    assert d < 1e-11 and abs(E - E0) <= 1e-11 * abs(E0)


def test_screening_keeps_the_dfma_kernel(ctx):
    """With pair screening the sliced form is not used: K equals the screened
    DFMA result bit for bit."""
    s = inputs.alkane_localised(30, lmax=2)
    tree, C = _build(ctx, s, 2)
    K1, E1 = _run(ctx, tree, C, 7, tau=1e-4)
    K0, E0 = _run(ctx, tree, C, 0, tau=1e-4)
    assert torch.equal(K1, K0) and E1 == E0


def test_slices_argument(ctx):
    from paper_1708_05353_gb300 import occk
    for bad in (-1, 1, 5, 8):
        with pytest.raises(occk.OcckError):
            ctx.set_fp64_slices(bad)


def test_sliced_per_edge_ranks(ctx):
    """Per-edge M2L ranks (lmax_policy 1): the double-FP32 M2L reads each
    edge's rank; K follows the oracle with the same ranks."""
    from oracle import fmm
    from oracle import tree as otree
    s = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    L = 4
    tr = otree.build_tree(s.basis, 3, 8.0)
    ranks = np.random.default_rng(3).integers(0, L + 1, size=len(tr["m2l_tgt"]))
    from paper_1708_05353_gb300 import occk
    tree = occk.Tree(ctx, s.basis, depth=3)
    tree.pair_multipoles(L)
    tree.set_edge_lmax(ranks)
    C = torch.tensor(s.C, dtype=torch.float64, device="cuda:0")
    ctx.set_fp64_slices(7)
    try:
        K, E = occk.farfield_K(ctx, tree, C, prec="fp64", lmax_policy=1, want_energy_host=True)
    finally:
        ctx.set_fp64_slices(0)
    Kr, Er = fmm.farfield(s, L=L, tree=tr, lmax_edges=ranks)
    err = rel_err(K.cpu().numpy(), Kr)
    print(f"per-edge ranks, 7 slices: {err:.2e}, |dE| {abs(E - Er):.2e}")
    assert err < 1e-11 and abs(E - Er) <= 1e-11 * abs(Er)


def test_sliced_learned_selector(ctx):
    """The learned selector (lmax_policy 2) reads the FP64 multipoles of every
    box: the sliced form joins its double-FP32 M2M's multipoles back to FP64
    for it, and at L = 6 runs the M2L from slices with the chosen ranks; with
    the same network the chosen ranks are the DFMA form's and K follows it."""
    from oracle import mlp
    from paper_1708_05353_gb300 import occk
    rng = np.random.default_rng(5)
    theta = mlp.init(occk.MLP_NIN, occk.MLP_HIDDEN, occk.MLP_NOUT, 5)
    norm = np.concatenate([rng.normal(size=occk.MLP_NIN), rng.uniform(0.5, 2.0, size=occk.MLP_NIN),
                           np.zeros(occk.MLP_NOUT), np.ones(occk.MLP_NOUT)])
    occk.mlp_set(ctx, theta, norm)
    s = inputs.alkane(30, lmax=6)
    tree, C = _build(ctx, s, 6)
    out = {}
    for sl in (0, 7):
        ctx.set_fp64_slices(sl)
        try:
            K, E = occk.farfield_K(ctx, tree, C, prec="fp64", lmax_policy=2, want_energy_host=True)
            out[sl] = (K.clone(), E, occk.edge_ranks(ctx, tree))
        finally:
            ctx.set_fp64_slices(0)
    (K0, E0, r0), (K7, E7, r7) = out[0], out[7]
    d = float((K7 - K0).abs().max() / K0.abs().max())
    print(f"learned ranks, 7 slices vs DFMA: {d:.2e}, |dE| {abs(E7 - E0):.2e}")
    assert np.array_equal(r0, r7)
    assert d < 1e-11 and abs(E7 - E0) <= 1e-11 * abs(E0)


@pytest.mark.parametrize("name,L", [("chain60", 6), ("chain20", 10)])
def test_sliced_m2l_matches_double_fp32(ctx, name, L):
    """M2L from slices (the default from L = 4) against the double-FP32 M2L
    of the same form: both are FP64-accurate, so K agrees far inside the
    slices' own truncation."""
    from paper_1708_05353_gb300 import occk
    s = inputs.alkane(60, lmax=L) if name == "chain60" else SYSTEMS["chain20"]()
    tree, C = _build(ctx, s, L)
    K1, E1 = _run(ctx, tree, C, 7)
    ctx.set_fp64_slice_m2l(False)
    try:
        K0, E0 = _run(ctx, tree, C, 7)
    finally:
        ctx.set_fp64_slice_m2l(True)
    d = float((K1 - K0).abs().max() / K0.abs().max())
    print(f"{name} L={L}: M2L from slices vs double-FP32 {d:.2e}, |dE| {abs(E1 - E0):.2e}")
    assert d < 1e-11 and abs(E1 - E0) <= 1e-12 * abs(E0)
    with pytest.raises(occk.OcckError):
        ctx.check(occk.lib().occk_set_fp64_slice_m2l(ctx._h, 2), "occk_set_fp64_slice_m2l")


def test_sliced_m2l_per_edge_ranks_match_double_fp32(ctx):
    """Per-edge ranks at L = 4: the M2L from slices uses each edge's
    operator restricted to its rank, like the double-FP32 M2L."""
    from oracle import tree as otree
    from paper_1708_05353_gb300 import occk
    s = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    L = 4
    tr = otree.build_tree(s.basis, 3, 8.0)
    ranks = np.random.default_rng(11).integers(0, L + 1, size=len(tr["m2l_tgt"]))
    tree = occk.Tree(ctx, s.basis, depth=3)
    tree.pair_multipoles(L)
    tree.set_edge_lmax(ranks)
    C = torch.tensor(s.C, dtype=torch.float64, device="cuda:0")
    out = {}
    ctx.set_fp64_slices(7)
    try:
        for on in (True, False):
            ctx.set_fp64_slice_m2l(on)
            K, E = occk.farfield_K(ctx, tree, C, prec="fp64", lmax_policy=1, want_energy_host=True)
            out[on] = (K.clone(), E)
    finally:
        ctx.set_fp64_slice_m2l(True)
        ctx.set_fp64_slices(0)
    d = float((out[True][0] - out[False][0]).abs().max() / out[False][0].abs().max())
    print(f"per-edge ranks: M2L from slices vs double-FP32 {d:.2e}")
    assert d < 1e-11 and abs(out[True][1] - out[False][1]) <= 1e-12 * abs(out[False][1])


def test_sliced_leaf_batches_are_bit_identical(ctx):
    """With a small slice workspace the leaves run in many batches (panels
    built and multiplied batch by batch), and so do the M2L's pair tiles;
    every output tile is computed the same way, so K and E are bit for bit
    those of one batch."""
    from paper_1708_05353_gb300 import occk
    s = SYSTEMS["chain60"]()
    tree, C = _build(ctx, s, 6)
    K1, E1 = _run(ctx, tree, C, 7)
    ctx.set_slice_workspace(48 << 20)
    try:
        K2, E2 = _run(ctx, tree, C, 7)
    finally:
        ctx.set_slice_workspace(0)
    assert torch.equal(K1, K2) and E1 == E2
    with pytest.raises(occk.OcckError):
        ctx.set_slice_workspace(-1)


def test_sliced_workspaces_are_released():
    """A context that ran the sliced form gives every workspace back when it
    is destroyed, and the form's panels when it is turned off.  (A first
    context runs the same build beforehand, so that the kernels' one-time
    loading is not counted.)"""
    from paper_1708_05353_gb300 import occk
    s = SYSTEMS["chain60"]()

    def run(off_first):
        c2 = occk.Context(0)
        tree, C = _build(c2, s, 6)
        c2.set_fp64_slices(7)
        occk.farfield_K(c2, tree, C, prec="fp64", want_energy_host=True)
        torch.cuda.synchronize()
        used = torch.cuda.mem_get_info()[0]
        c2.set_fp64_slices(0)
        off = torch.cuda.mem_get_info()[0]
        tree.close()
        c2.close()
        del C
        torch.cuda.empty_cache()
        return used, off

    run(True)
    free0 = torch.cuda.mem_get_info()[0]
    used, off = run(True)
    free1 = torch.cuda.mem_get_info()[0]
    print(f"free GB: before {free0 / 1e9:.3f}, in use {used / 1e9:.3f}, form off {off / 1e9:.3f}, "
          f"closed {free1 / 1e9:.3f}")
    assert off > used + (64 << 20)             # the panels (several hundred MB here) came back
    assert abs(free1 - free0) <= (64 << 20)
