"""The failure path of the bounded device waits, made to run on purpose.

Every wait of the tensor-core kernels on an mbarrier is bounded.  Here the
MMA-issuing thread of the panel GEMMs (steps (a) and (e) of the mixed forms
and of the integer-slice forms) is allowed zero polls for its operands, so its first wait gives up: the
kernel raises its abort flag, waits with the normal limit for the bulk copies
and MMAs it has in flight, frees its TMEM and returns, and the host reads the
device error word.  Nothing faults, traps or hangs: the wait that gives up is
one whose copies do land, only later.  The call must report OCCK_ERR_TIMEOUT,
and the next call with the default limit must give the same K and E as a
clean run (the context stays usable).
"""
import numpy as np
import pytest

from paper_1708_05353_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    from paper_1708_05353_gb300 import occk
    ctx = occk.Context(0)
    s = inputs.water(nmol=12, lmax=4)
    tree = occk.Tree(ctx, s.basis, depth=2)
    tree.pair_multipoles(4)
    C = torch.tensor(s.C, dtype=torch.float64, device="cuda:0")
    yield occk, ctx, tree, s, C
    ctx.debug_set_wait_limit(-1)


@pytest.mark.parametrize("prec", ["fp16x3", "tf32"])
def test_wait_gives_up_then_context_recovers(setup, prec):
    occk, ctx, tree, s, C = setup
    K0, E0 = occk.farfield_K(ctx, tree, C, prec=prec, want_energy_host=True)
    K0 = K0.cpu().numpy()
    ctx.debug_set_wait_limit(0)
    try:
        with pytest.raises(occk.OcckError) as e:
            occk.farfield_K(ctx, tree, C, prec=prec, want_energy_host=True)
        assert e.value.code == -5, str(e.value)
        with pytest.raises(occk.OcckError) as e2:
            occk.device_status(ctx)
        assert e2.value.code == -5
    finally:
        ctx.debug_set_wait_limit(-1)
    K1, E1 = occk.farfield_K(ctx, tree, C, prec=prec, want_energy_host=True)
    occk.device_status(ctx)                     # clean again
    assert np.array_equal(K1.cpu().numpy(), K0) and E1 == E0


@pytest.mark.parametrize("form", ["fp64s", "fp32s"])
def test_slice_gemm_wait_gives_up_then_recovers(setup, form):
    """The same failure path in the integer-slice GEMMs (steps (a) and (e) of
    the FP64-accurate and FP32 slice forms): an abort in the middle of an
    accumulation chunk still waits for the MMAs it issued before TMEM is
    freed, and the context gives the clean result afterwards."""
    occk, ctx, tree, s, C = setup
    prec = "fp64" if form == "fp64s" else "fp32"
    setter = ctx.set_fp64_slices if form == "fp64s" else ctx.set_fp32_slices
    setter(7 if form == "fp64s" else 4)
    try:
        K0, E0 = occk.farfield_K(ctx, tree, C, prec=prec, want_energy_host=True)
        K0 = K0.cpu().numpy()
        ctx.debug_set_wait_limit(0)
        try:
            with pytest.raises(occk.OcckError) as e:
                occk.farfield_K(ctx, tree, C, prec=prec, want_energy_host=True)
            assert e.value.code == -5, str(e.value)
        finally:
            ctx.debug_set_wait_limit(-1)
        K1, E1 = occk.farfield_K(ctx, tree, C, prec=prec, want_energy_host=True)
        occk.device_status(ctx)
        assert np.array_equal(K1.cpu().numpy(), K0) and E1 == E0
    finally:
        setter(0)


def test_debug_gemm_wait_gives_up(setup):
    occk, ctx, tree, s, C = setup
    g = torch.Generator(device="cpu").manual_seed(3)
    A = torch.randn(200, 300, generator=g).float().cuda()
    B = torch.randn(150, 300, generator=g).float().cuda()
    ctx.debug_set_wait_limit(0)
    try:
        with pytest.raises(occk.OcckError) as e:
            occk.debug_tc_gemm(ctx, "fp16x3", A, B)
        assert e.value.code == -5
    finally:
        ctx.debug_set_wait_limit(-1)
    D = occk.debug_tc_gemm(ctx, "fp16x3", A, B)
    ref = (A.double() @ B.double().T)
    assert float((D.double() - ref).abs().max() / ref.abs().max()) < 2e-6
