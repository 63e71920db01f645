"""The Python binding rejects operands that the C ABI cannot check.

The C entry points receive bare device pointers and sizes; a K with fewer
columns than C, a float32 tensor where float64 is required, or a tensor on
another device would make a kernel read or write outside the buffer.  The
binding therefore checks dtype, shape and device of every tensor before the
library is called, and raises OcckError (ERR_ARG for dtype/device, ERR_SHAPE
for shape).  The CPU tests use a host-only context (no kernel can run there);
the GPU tests repeat the shape checks on device tensors.
"""
import numpy as np
import pytest

from paper_1708_05353_gb300 import inputs

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def host():
    from paper_1708_05353_gb300 import occk
    ctx = occk.Context(-1)
    s = inputs.small_sp(natom=4, nocc=3, spacing=3.0, depth=2)
    tree = occk.Tree(ctx, s.basis, depth=2)
    return occk, ctx, tree, s


def _code(fn):
    from paper_1708_05353_gb300 import occk
    with pytest.raises(occk.OcckError) as e:
        fn()
    return e.value.code, str(e.value)


def test_farfield_K_rejects_bad_operands(host):
    occk, ctx, tree, s = host
    nao, nocc = s.basis.nao, s.nocc
    C32 = torch.zeros(nao, nocc, dtype=torch.float32)
    assert _code(lambda: occk.farfield_K(ctx, tree, C32))[0] == -1
    Cbad = torch.zeros(nao + 1, nocc, dtype=torch.float64)
    assert _code(lambda: occk.farfield_K(ctx, tree, Cbad))[0] == -2
    C = torch.zeros(nao, nocc, dtype=torch.float64)
    code, msg = _code(lambda: occk.farfield_K(ctx, tree, C))
    assert code == -1 and "cuda" in msg
    # K with fewer columns than C, K in float32, a 1-element energy buffer
    Ksmall = torch.zeros(nao, nocc - 1, dtype=torch.float64)
    assert _code(lambda: occk.farfield_K(ctx, tree, C, K=Ksmall))[0] == -2
    K32 = torch.zeros(nao, nocc, dtype=torch.float32)
    assert _code(lambda: occk.farfield_K(ctx, tree, C, K=K32))[0] == -1
    K = torch.zeros(nao, nocc, dtype=torch.float64)
    E1 = torch.zeros(1, dtype=torch.float64)
    assert _code(lambda: occk.farfield_K(ctx, tree, C, K=K, Ex=E1))[0] in (-1, -2)


def test_noalloc_energy_rejects_bad_operands(host):
    occk, ctx, tree, s = host
    C = torch.zeros(5, 3, dtype=torch.float64)
    assert _code(lambda: occk.exchange_energy_noalloc(ctx, C, torch.zeros(5, 2, dtype=torch.float64)))[0] == -2
    assert _code(lambda: occk.exchange_energy_noalloc(ctx, C, torch.zeros(5, 3, dtype=torch.float32)))[0] == -1
    assert _code(lambda: occk.exchange_energy_noalloc(ctx, C.float(), C.float()))[0] == -1
    E32 = torch.zeros((), dtype=torch.float32)
    assert _code(lambda: occk.exchange_energy_noalloc(ctx, C, C.clone(), E32))[0] == -1
    # right dtypes and shapes, but host memory: refused before the call
    assert _code(lambda: occk.exchange_energy_noalloc(ctx, C, C.clone()))[0] == -1


def test_farfield_J_rejects_bad_operands(host):
    occk, ctx, tree, s = host
    nao = s.basis.nao
    assert _code(lambda: occk.farfield_J(ctx, tree, torch.zeros(nao, nao - 1, dtype=torch.float64)))[0] == -2
    assert _code(lambda: occk.farfield_J(ctx, tree, torch.zeros(nao, nao, dtype=torch.float32)))[0] == -1


@pytest.mark.gpu
def test_device_operands_checked_before_launch():
    from paper_1708_05353_gb300 import occk
    ctx = occk.Context(0)
    s = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    tree = occk.Tree(ctx, s.basis, depth=3)
    tree.pair_multipoles(2)
    C = torch.tensor(s.C, dtype=torch.float64, device="cuda:0")
    Ksmall = occk.empty_fortran(s.basis.nao, s.nocc - 1, torch.float64, "cuda:0")
    assert _code(lambda: occk.farfield_K(ctx, tree, C, K=Ksmall))[0] == -2
    K, E = occk.farfield_K(ctx, tree, C)
    assert _code(lambda: occk.exchange_energy_noalloc(ctx, occk.fortran(C), Ksmall))[0] == -2
    assert _code(lambda: occk.exchange_energy_noalloc(ctx, occk.fortran(C), K.float()))[0] == -1
    torch.cuda.synchronize()
    assert np.isfinite(float(E.item()))
