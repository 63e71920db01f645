"""GPU parity of the far-field Coulomb matrix (Sec. II: density multipoles,
Eq. fmmc, and J^ff_rs = sum_lm O^{rs,X}_lm Mcal_lm(X)) through the C ABI
against the FP64 oracle, which its own tests tie to exact far-box four-centre
integrals.  Bar: the plain-FP64 one, max|dJ|/max|J| <= 1e-10 and
|dE_J|/|E_J| <= 1e-10.  For one occupied orbital the Coulomb and exchange far
fields come from the same bilinear approximation of (rs|tu), so the CUDA
paths must give E_J = -2 E_K to rounding."""
import numpy as np
import pytest

from oracle import fmm_j
from oracle import tree as otree
from paper_1708_05353_gb300 import inputs
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_1708_05353_gb300 import occk
    return occk.Context(0)


def _density(C):
    return 2.0 * C @ C.T


def _gpu(ctx, s, L, depth=None):
    from paper_1708_05353_gb300 import occk
    d = s.depth if depth is None else depth
    tree = occk.Tree(ctx, s.basis, depth=d, target_atoms_per_leaf=s.target_atoms_per_leaf)
    tree.pair_multipoles(L)
    D = torch.tensor(_density(s.C), dtype=torch.float64, device="cuda:0")
    J, E = occk.farfield_J(ctx, tree, D, want_energy_host=True)
    torch.cuda.synchronize()
    return tree, J.cpu().numpy(), E


def _oracle(s, L, depth=None):
    d = s.depth if depth is None else depth
    tr = otree.build_tree(s.basis, d, s.target_atoms_per_leaf)
    return fmm_j.farfield_J(s.basis, _density(s.C), L, tr)


@pytest.mark.parametrize("L", [0, 1, 2, 3, 6])
def test_j_fp64_small_sp(ctx, L):
    s = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    _, J, E = _gpu(ctx, s, L)
    Jr, Er = _oracle(s, L)
    assert rel_err(J, Jr) < 1e-10
    assert abs(E - Er) <= 1e-10 * abs(Er)


@pytest.mark.parametrize("L", [2, 6])
def test_j_fp64_line40(ctx, L):
    """40 hydrogens on a line, depth 4: M2M and L2L over two levels."""
    s = inputs.tiny_line()
    _, J, E = _gpu(ctx, s, L)
    Jr, Er = _oracle(s, L)
    assert rel_err(J, Jr) < 1e-10
    assert abs(E - Er) <= 1e-10 * abs(Er)


def test_j_fp64_water_3d(ctx):
    """3-D cluster with s and p shells, every leaf with several pairs."""
    s = inputs.water(nmol=12, lmax=4)
    _, J, E = _gpu(ctx, s, 4, depth=2)
    Jr, Er = _oracle(s, 4, depth=2)
    assert rel_err(J, Jr) < 1e-10
    assert abs(E - Er) <= 1e-10 * abs(Er)


def test_j_symmetric_and_zero_off_pairs(ctx):
    """J is symmetric to rounding: within one shell pair (r, s) and (s, r)
    read the multipoles O^{rs} and O^{sr}, equal but computed separately."""
    s = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    _, J, _ = _gpu(ctx, s, 3)
    Jr, _ = _oracle(s, 3)
    assert np.max(np.abs(J - J.T)) <= 1e-13 * np.max(np.abs(J))
    assert np.all(J[Jr == 0] == 0)


@pytest.mark.parametrize("L", [0, 3, 5])
def test_j_minus_twice_k_one_orbital(ctx, L):
    from paper_1708_05353_gb300 import occk
    s = inputs.small_sp(natom=6, nocc=1, spacing=3.0, depth=3)
    tree, _, EJ = _gpu(ctx, s, L)
    C = torch.tensor(s.C, dtype=torch.float64, device="cuda:0")
    _, EK = occk.farfield_K(ctx, tree, C, prec="fp64", want_energy_host=True)
    assert abs(EJ + 2.0 * EK) <= 1e-12 * abs(EJ)


def test_j_no_far_field(ctx):
    """Depth 1: no interaction lists, J^ff = 0 and E_J = 0."""
    s = inputs.small_sp(natom=4, nocc=2, spacing=3.0, depth=1)
    _, J, E = _gpu(ctx, s, 2, depth=1)
    assert np.all(J == 0) and E == 0.0


def test_j_strided_and_repeatable(ctx):
    """Leading dimensions larger than nao, and the same call twice gives
    bit-identical results."""
    from paper_1708_05353_gb300 import occk
    s = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    tree, J1, E1 = _gpu(ctx, s, 4)
    n = s.basis.nao
    Dbig = torch.zeros((n + 5, n), dtype=torch.float64, device="cuda:0")
    Dbig[:n] = torch.tensor(_density(s.C), dtype=torch.float64, device="cuda:0")
    Dv = Dbig.t().contiguous().t()[:n]          # column-major, ld = n + 5
    Jbig = torch.full((n, n + 3), 7.0, dtype=torch.float64, device="cuda:0").t()   # ld = n + 3
    Jv = Jbig[:n]
    J2, E2 = occk.farfield_J(ctx, tree, Dv, J=Jv, want_energy_host=True)
    torch.cuda.synchronize()
    assert E1 == E2
    assert np.array_equal(J2.cpu().numpy(), J1)
    assert torch.all(Jbig[n:] == 7.0)
