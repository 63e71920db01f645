"""Pins of the far-field Coulomb oracle (Sec. II, Eq. fmmc and the J^ff
formula): convergence in the rank to the exact far-box four-centre result on
s-only and s/p systems, symmetry, and, for one occupied orbital, the identity
E_J = -2 E_K that holds rank by rank because both use the same bilinear
far-field approximation of (rs|tu)."""
import numpy as np
import pytest

from oracle import fmm, fmm_j
from oracle import tree as otree
from paper_1708_05353_gb300 import inputs


def _density(C):
    return 2.0 * C @ C.T


@pytest.mark.parametrize("kind", ["line", "sp"])
def test_j_converges_to_exact(kind):
    s = inputs.tiny_line() if kind == "line" else inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    tr = otree.build_tree(s.basis, s.depth, s.target_atoms_per_leaf)
    D = _density(s.C)
    Jx, Ex = fmm_j.farfield_J_exact(s.basis, tr, D)
    errs = []
    for L in (1, 3, 6):
        J, E = fmm_j.farfield_J(s.basis, D, L, tr)
        errs.append(np.max(np.abs(J - Jx)) / np.max(np.abs(Jx)))
        assert abs(E - 0.5 * np.sum(D * J)) < 1e-12
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 1e-3


def test_j_symmetric_and_real():
    s = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    tr = otree.build_tree(s.basis, s.depth, s.target_atoms_per_leaf)
    J, _ = fmm_j.farfield_J(s.basis, _density(s.C), 4, tr)
    assert np.allclose(J, J.T, rtol=0, atol=1e-14)
    assert np.max(np.abs(J)) > 0


@pytest.mark.parametrize("L", [0, 2, 5])
def test_one_orbital_coulomb_is_minus_twice_exchange(L):
    s = inputs.small_sp(natom=6, nocc=1, spacing=3.0, depth=3)
    tr = otree.build_tree(s.basis, s.depth, s.target_atoms_per_leaf)
    _, EK = fmm.farfield(s, L=L, tree=tr)
    _, EJ = fmm_j.farfield_J(s.basis, _density(s.C), L, tr)
    assert abs(EJ + 2.0 * EK) <= 1e-12 * abs(EJ)
