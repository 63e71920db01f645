"""The library's occupied column-block mode (one rank's share of a sharded
build) on one GPU: the blocks of two or three ranks, computed one after the
other through occk_set_column_block and put together, give the unblocked
K bit for bit in FP64 and FP32 (every pair's multipoles and local expansions
are computed by the same arithmetic whichever pairs are kept, and each K
column sums the same terms in the same order), occk_exchange_energy on the
assembled K gives the unblocked E bit for bit, and each block's own energy
is its part of E.  The tensor-core forms follow within their bounds.
The ranks are run one after another: nothing here waits on another rank.
"""
import numpy as np
import pytest

from paper_1708_05353_gb300 import inputs, shard

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_1708_05353_gb300 import occk
    c = occk.Context(0)
    yield c
    c.set_column_block(0, 0)


def _setup(ctx, s, L):
    from paper_1708_05353_gb300 import occk
    tree = occk.Tree(ctx, s.basis, depth=s.depth, target_atoms_per_leaf=s.target_atoms_per_leaf)
    tree.pair_multipoles(L)
    C = occk.fortran(torch.tensor(s.C, dtype=torch.float64, device="cuda:0"))
    return tree, C


def _blocks_run(ctx, tree, C, blocks, prec):
    from paper_1708_05353_gb300 import occk
    nao, nocc = C.shape
    Kall = occk.empty_fortran(nao, nocc, torch.float64, "cuda:0")
    Kall.fill_(float("nan"))
    parts = []
    for c0, c1 in blocks:
        ctx.set_column_block(c0, c1)
        try:
            K, E = occk.farfield_K(ctx, tree, C, prec=prec, want_energy_host=True)
        finally:
            ctx.set_column_block(0, 0)
        Kall[:, c0:c1] = K[:, c0:c1]
        parts.append(E)
    return Kall, parts


@pytest.mark.parametrize("name,L,world", [("chain60", 2, 2), ("chain60", 2, 3), ("water", 4, 2)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_blocks_reproduce_unblocked_bit_for_bit(ctx, name, L, world, prec):
    from paper_1708_05353_gb300 import occk
    s = inputs.alkane(60, lmax=L) if name == "chain60" else inputs.water(nmol=12, lmax=L)
    if name == "water":
        s.depth = 2
    tree, C = _setup(ctx, s, L)
    K0, E0 = occk.farfield_K(ctx, tree, C, prec=prec, want_energy_host=True)
    blocks = shard.column_blocks(s.nocc, world)
    Kall, parts = _blocks_run(ctx, tree, C, blocks, prec)
    assert torch.equal(Kall, K0)
    E = occk.exchange_energy(ctx, C, Kall)
    assert float(E.item()) == E0
    C_h, K_h = s.C, K0.cpu().numpy()
    for (c0, c1), Eb in zip(blocks, parts):
        ref = -0.5 * float(np.sum(C_h[:, c0:c1] * K_h[:, c0:c1]))
        assert abs(Eb - ref) <= 1e-12 * abs(E0)


@pytest.mark.parametrize("prec", ["fp16x3", "tf32"])
def test_blocks_tensor_core_forms(ctx, prec):
    from paper_1708_05353_gb300 import occk
    s = inputs.alkane(60, lmax=2)
    tree, C = _setup(ctx, s, 2)
    K64, E64 = occk.farfield_K(ctx, tree, C, prec="fp64", want_energy_host=True)
    Kall, _ = _blocks_run(ctx, tree, C, shard.column_blocks(s.nocc, 2), prec)
    bound = {"fp16x3": 1e-5, "tf32": 1e-2}[prec]
    assert float((Kall - K64).abs().max() / K64.abs().max()) < bound


def test_block_argument_checks(ctx):
    from paper_1708_05353_gb300 import occk
    s = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    tree, C = _setup(ctx, s, 2)
    with pytest.raises(occk.OcckError):
        ctx.set_column_block(3, 2)
    ctx.set_column_block(2, 9)
    try:
        with pytest.raises(occk.OcckError) as e:
            occk.farfield_K(ctx, tree, C)
        assert e.value.code == -2
    finally:
        ctx.set_column_block(0, 0)


def test_sharded_driver_single_rank(ctx):
    """farfield_K_sharded with one rank is the plain call."""
    from paper_1708_05353_gb300 import occk
    s = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    tree, C = _setup(ctx, s, 3)
    K0, E0 = occk.farfield_K(ctx, tree, C, want_energy_host=True)
    K, E = shard.farfield_K_sharded(ctx, tree, C, shard.column_blocks(s.nocc, 1), 0)
    assert torch.equal(K, K0) and float(E.item()) == E0
