"""Mixed-precision tensor-core forms against FP64 references.

The engine (tcgen05 MMA, TMEM accumulator, hi/lo operand splitting) is first
checked on plain GEMMs with ragged shapes against an FP64 product; then the
far-field exchange in each precision is checked against the FP64 oracle with
a per-precision bound.  The bounds follow from the input formats: one product
of two values rounded to p significant bits has relative error <= 2^-p
(BF16 p=8, FP16 and TF32 p=11); the split forms drop only the lo*lo term,
about 2^-2p; FP32 accumulation adds ~K * 2^-24.
"""
import numpy as np
import pytest

from oracle import fmm
from oracle import tree as otree
from paper_1708_05353_gb300 import inputs
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GEMM_BOUND = {"bf16": 2e-2, "fp16": 4e-3, "tf32": 4e-3, "bf16x3": 1e-4, "fp16x3": 2e-6}
K_BOUND = {"bf16": 5e-2, "fp16": 1e-2, "tf32": 1e-2, "bf16x3": 1e-3, "fp16x3": 1e-5}


@pytest.fixture(scope="module")
def ctx():
    from paper_1708_05353_gb300 import occk
    return occk.Context(0)


@pytest.mark.parametrize("prec", list(GEMM_BOUND))
@pytest.mark.parametrize("shape", [(128, 128, 64), (200, 150, 100), (37, 300, 259)])
def test_tc_gemm(ctx, prec, shape):
    from paper_1708_05353_gb300 import occk
    M, N, K = shape
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g, dtype=torch.float32).cuda()
    B = torch.randn(N, K, generator=g, dtype=torch.float32).cuda()
    D = occk.debug_tc_gemm(ctx, prec, A, B)
    torch.cuda.synchronize()
    ref = (A.double() @ B.double().T).cpu().numpy()
    err = rel_err(D.cpu().double().numpy(), ref)
    print(f"tc gemm {prec} {shape}: rel err {err:.2e}")
    assert err < GEMM_BOUND[prec]


@pytest.fixture(scope="module")
def water_ref():
    s = inputs.water(nmol=12, lmax=4)
    tr = otree.build_tree(s.basis, 2, 8.0)
    K, E = fmm.farfield(s, L=4, tree=tr)
    return s, K, E


@pytest.mark.parametrize("prec", ["fp32"] + list(K_BOUND))
def test_mixed_farfield_water(ctx, water_ref, prec):
    from paper_1708_05353_gb300 import occk
    s, Kr, Er = water_ref
    tree = occk.Tree(ctx, s.basis, depth=2)
    tree.pair_multipoles(4)
    C = torch.tensor(s.C, dtype=torch.float64, device="cuda:0")
    K, E = occk.farfield_K(ctx, tree, C, prec=prec, want_energy_host=True)
    Kg = K.cpu().numpy()
    err = rel_err(Kg, Kr)
    print(f"far field {prec}: max|dK|/max|K| = {err:.2e}, |dE| = {abs(E - Er):.2e} Eh (E = {Er:.8f})")
    assert err < K_BOUND.get(prec, 1e-4)
    assert abs(E - Er) <= K_BOUND.get(prec, 1e-4) * abs(Er)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tc_integer_products_exact(ctx, prec):
    """Sums of products of small integers are exact on the tensor core: with
    |a|, |b| <= 64 every product is an integer below 2^12 and every partial
    sum below 2^24, so the FP32 accumulation (in TMEM within a stage, in
    registers across stages) rounds nothing; mixed magnitudes within one MMA
    (1 next to 64) lose no low bits either."""
    from paper_1708_05353_gb300 import occk
    g = torch.Generator(device="cpu").manual_seed(5)
    K = 2048
    A = torch.randint(-64, 65, (256, K), generator=g)
    B = torch.randint(-64, 65, (192, K), generator=g)
    A[:8] = 64                                          # worst case: K * 64 * 64 = 2^23
    B[:8] = 64
    A[8:16, ::2] = 1                                    # small next to large in every K step
    ref = A.double() @ B.double().T
    D = occk.debug_tc_gemm(ctx, prec, A.float().cuda(), B.float().cuda()).double().cpu()
    assert float(ref.abs().max()) == 2.0 ** 23
    assert torch.equal(D, ref)


@pytest.mark.parametrize("prec,bound", [("fp16x3", 5e-7), ("bf16x3", 2e-6), ("tf32", 2e-5)])
def test_tc_long_sum_unbiased(ctx, prec, bound):
    """The tensor core's FP32 accumulation is biased toward zero over long
    chains; the engine restarts the accumulator every stage and sums stages in
    FP32 registers, so a K = 8192 sum of positive products stays unbiased to
    the level of its operand rounding."""
    from paper_1708_05353_gb300 import occk
    g = torch.Generator(device="cpu").manual_seed(11)
    A = (1.0 + 0.1 * torch.rand(128, 8192, generator=g)).float().cuda()
    B = (1.0 + 0.1 * torch.rand(128, 8192, generator=g)).float().cuda()
    D = occk.debug_tc_gemm(ctx, prec, A, B).double()
    ref = A.double() @ B.double().T
    bias = float(((D - ref) / ref).mean())
    print(f"{prec}: mean relative error over K = 8192: {bias:.2e}")
    assert abs(bias) < bound
