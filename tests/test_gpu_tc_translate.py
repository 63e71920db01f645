"""Tensor-core translations of the mixed forms: M2M, M2L and L2L on tcgen05
(Eqs. fmm1-3), checked against the FP64 path on the same tree and against
exact K columns of the FP64 oracle (tests/golden/oracle_columns.npz, written
by tests/golden/make_columns.py from the oracle alone).

Every expansion order that selects a different GEMM width (L = 2, 4, 6, 10:
N = 16, 32, 64, 128) runs on an alkane chain deep enough for M2M and L2L, with
81 occupied orbitals, so 3321 stored pairs: 25 full pair tiles and a ragged
one.  The bounds are those of the mixed forms' GEMMs (one rounding of each
operand to p bits, 2^-p relative per product; split forms ~2^-2p) with the
same allowance for accumulation over a few hundred terms as for steps (a) and
(e).  The local expansions of every box are compared too, so an error in one
translation kind cannot hide behind the others.
"""
import os

import numpy as np
import pytest

from paper_1708_05353_gb300 import inputs
from tests.helpers import rel_err

GOLD = np.load(os.path.join(os.path.dirname(__file__), "golden", "oracle_columns.npz"))

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

K_BOUND = {"bf16": 5e-2, "fp16": 1e-2, "tf32": 1e-2, "bf16x3": 1e-3, "fp16x3": 1e-5}


@pytest.fixture(scope="module")
def ctx():
    from paper_1708_05353_gb300 import occk
    c = occk.Context(0)
    c.set_translate_engine(7)      # all three translations on the tensor core
    return c


@pytest.fixture(scope="module")
def chain():
    return inputs.alkane(20, lmax=10, seed_k=4)


def _tree(ctx, s, L):
    from paper_1708_05353_gb300 import occk
    t = occk.Tree(ctx, s.basis, depth=s.depth, target_atoms_per_leaf=s.target_atoms_per_leaf)
    t.pair_multipoles(L)
    return t


def _run(ctx, tree, s, prec, policy=0):
    from paper_1708_05353_gb300 import occk
    C = torch.tensor(s.C, dtype=torch.float64, device="cuda:0")
    K, E = occk.farfield_K(ctx, tree, C, prec=prec, lmax_policy=policy, want_energy_host=True)
    torch.cuda.synchronize()
    return K.cpu().numpy(), E


@pytest.mark.parametrize("engine", [7, 15])
@pytest.mark.parametrize("L", [2, 4, 6, 10])
@pytest.mark.parametrize("prec", list(K_BOUND))
def test_tc_translate_chain(ctx, chain, L, prec, engine):
    """engine 7: operands converted in registers at every use; engine 15:
    expansions kept in the tensor core's layout (slots) between the steps."""
    from paper_1708_05353_gb300 import occk
    s = chain
    tree = _tree(ctx, s, L)
    assert tree.info()["depth"] >= 3          # M2M and L2L both run
    K64, E64 = _run(ctx, tree, s, "fp64")
    M64 = occk.debug_fetch(ctx, tree, "mbox", nocc=s.nocc, stream=0)
    ctx.set_translate_engine(engine)
    try:
        K, E = _run(ctx, tree, s, prec)
        M = occk.debug_fetch(ctx, tree, "mbox", nocc=s.nocc, stream=0)
    finally:
        ctx.set_translate_engine(7)
    errK = rel_err(K, K64)
    errM = max(rel_err(M[b], M64[b]) for b in range(M.shape[0]) if np.abs(M64[b]).max() > 0)
    cols = GOLD["chain20/cols"]
    fp = GOLD["chain20/fingerprint"]
    assert [s.basis.nao, s.nocc, tree.info()["nm2l"]] == [int(fp[0]), int(fp[1]), int(fp[4])]
    errO = rel_err(K[:, cols], GOLD[f"chain20/L{L}/K"])
    err64 = rel_err(K64[:, cols], GOLD[f"chain20/L{L}/K"])
    print(f"L={L} {prec} engine {engine}: K {errK:.2e} (oracle columns {errO:.2e}; FP64 path {err64:.2e}), "
          f"Mcal {errM:.2e}, |dE| {abs(E - E64):.2e} (E = {E64:.6f})")
    assert err64 < 1e-10
    assert errO < K_BOUND[prec]
    assert errK < K_BOUND[prec]
    assert errM < 4 * K_BOUND[prec]
    assert abs(E - E64) <= K_BOUND[prec] * abs(E64)


@pytest.mark.parametrize("engine", [7, 15])
def test_tc_translate_fp16x3_meets_energy_target(ctx, chain, engine):
    """The split FP16 form stays within 1e-6 Eh of the FP64 exchange energy
    at the highest order, where the operands span the widest range."""
    s = chain
    tree = _tree(ctx, s, 10)
    _, E64 = _run(ctx, tree, s, "fp64")
    ctx.set_translate_engine(engine)
    try:
        _, E = _run(ctx, tree, s, "fp16x3")
    finally:
        ctx.set_translate_engine(7)
    assert abs(E - E64) < 1e-6


def test_tc_translate_with_edge_ranks(ctx, chain):
    """Per-edge ranks keep M2L on the SIMT form (the truncated operator differs
    per edge) while M2M and L2L stay on the tensor core; the result must still
    follow the FP64 path with the same ranks."""
    s = chain
    L = 6
    tree = _tree(ctx, s, L)
    n = tree.info()["nm2l"]
    ranks = np.random.default_rng(5).integers(2, L + 1, size=n).astype(np.int32)
    tree.set_edge_lmax(ranks)
    K64, E64 = _run(ctx, tree, s, "fp64", policy=1)
    K, E = _run(ctx, tree, s, "fp16x3", policy=1)
    assert rel_err(K, K64) < K_BOUND["fp16x3"]
    assert abs(E - E64) <= K_BOUND["fp16x3"] * abs(E64)


@pytest.mark.parametrize("mask", [0, 2, 5])
def test_tc_translate_engine_mix(ctx, chain, mask):
    """Any mix of tensor-core and SIMT translations on the scaled storage
    (mask 2: M2L on the tensor core, M2M and L2L on SIMT with the scaled
    operators; mask 5 the other way round; mask 0: all SIMT, unscaled) gives
    the same far field."""
    s = chain
    tree = _tree(ctx, s, 6)
    K64, E64 = _run(ctx, tree, s, "fp64")
    ctx.set_translate_engine(mask)
    try:
        K, E = _run(ctx, tree, s, "fp16x3")
    finally:
        ctx.set_translate_engine(7)
    assert rel_err(K, K64) < K_BOUND["fp16x3"]
    assert abs(E - E64) <= K_BOUND["fp16x3"] * abs(E64)


@pytest.mark.parametrize("engine", [7, 15])
def test_tc_translate_repeatable(ctx, chain, engine):
    """The same call twice gives bit-identical results (no race between the
    pair tiles or between the CTAs that share a target)."""
    s = chain
    tree = _tree(ctx, s, 4)
    ctx.set_translate_engine(engine)
    try:
        K1, E1 = _run(ctx, tree, s, "fp16x3")
        K2, E2 = _run(ctx, tree, s, "fp16x3")
    finally:
        ctx.set_translate_engine(7)
    assert np.array_equal(K1, K2) and E1 == E2
