"""The allocation-free energy entry point against the regular path.

occk_exchange_energy_noalloc serves callers that cannot let the library call
cudaMalloc (their own allocator owns device memory, or an allocation would
stall a latency-sensitive loop).  Its scratch is a static device array, so
this test checks that two calls in a row -- the second reusing whatever the
first left in that array -- both reproduce the energy that occk_farfield_K
computes from the same K and C, within the FP64 tolerance of the other GPU
tests (1e-10 relative).  The file is named to run last.
"""
import numpy as np
import pytest

from paper_1708_05353_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _farfield(ctx, s, L, depth):
    from paper_1708_05353_gb300 import occk
    tree = occk.Tree(ctx, s.basis, depth=depth)
    tree.pair_multipoles(L)
    C = occk.fortran(torch.tensor(s.C, dtype=torch.float64, device="cuda:0"))
    K, E = occk.farfield_K(ctx, tree, C)
    return tree, C, K, E


@pytest.mark.parametrize("which", ["sp", "water"])
def test_noalloc_energy_matches_farfield(which):
    from paper_1708_05353_gb300 import occk
    ctx = occk.Context(0)
    if which == "sp":
        s, L, depth = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3), 3, 3
    else:
        s, L, depth = inputs.water(nmol=12, lmax=4), 4, 2
    tree, C, K, E_ref = _farfield(ctx, s, L, depth)
    torch.cuda.synchronize()
    e_ref = float(E_ref.item())
    assert e_ref != 0.0
    E = torch.empty((), dtype=torch.float64, device="cuda:0")
    for _ in range(2):
        E.fill_(np.nan)
        occk.exchange_energy_noalloc(ctx, C, K, E)
        torch.cuda.synchronize()
        assert abs(float(E.item()) - e_ref) <= 1e-10 * abs(e_ref)


def test_noalloc_rejects_oversize():
    from paper_1708_05353_gb300 import occk
    ctx = occk.Context(0)
    nao, nocc = 4, 8193
    C = occk.empty_fortran(nao, nocc, torch.float64, "cuda:0")
    with pytest.raises(occk.OcckError) as e:
        occk.exchange_energy_noalloc(ctx, C, C)
    assert e.value.code == -2
    assert "OCCK_NOALLOC_MAX_OCC" in str(e.value)
