"""Pins of the oracle's occupied-pair screening (the paper's proposed
extension to localised orbitals, Sec. IV).  Pairs are independent in the tree
passes and in K, so the far-field energy is a sum of pair energies
e_ij = -sum_X sum_lm O^{ij,X}_lm Mcal^{ij}_lm(X); dropping a set of pairs must
change E by exactly the sum of their e_ij taken from the unscreened run.
Also: tau = 0 is the unscreened method, a tau above every pair norm leaves
no far field, diagonal pairs (Sum_X O^{ii}_00 = 1 for orthonormal orbitals)
survive any tau^2 < 1/nleaf, and localised orbitals leave most pairs
negligible at a small energy change."""
import numpy as np
import pytest

from oracle import fmm
from oracle import tree as otree
from paper_1708_05353_gb300 import inputs
from tests.helpers import tau_in_gap


@pytest.fixture(scope="module")
def loc():
    s = inputs.small_sp_localised()
    tr = otree.build_tree(s.basis, s.depth, s.target_atoms_per_leaf)
    K0, E0, parts = fmm.farfield(s, L=3, tree=tr, return_parts=True)
    return s, tr, K0, E0, parts


def _pair_energies(tr, parts):
    lo = tr["level_off"][tr["depth"]]
    O = parts["Obox"][lo:]
    M = parts["Mbox"][lo:]
    return -np.real(np.einsum("xlij,xlij->ij", O, M))


def test_pair_energies_sum_to_energy(loc):
    s, tr, K0, E0, parts = loc
    e = _pair_energies(tr, parts)
    assert abs(e.sum() - E0) <= 1e-12 * abs(E0)


def test_tau_zero_is_unscreened(loc):
    s, tr, K0, E0, _ = loc
    K, E = fmm.farfield(s, L=3, tree=tr, pair_tau=0.0)
    assert np.array_equal(K, K0) and E == E0


@pytest.mark.parametrize("q", [0.3, 0.6, 0.85])
def test_screened_energy_is_minus_dropped_pairs(loc, q):
    s, tr, K0, E0, parts = loc
    e = _pair_energies(tr, parts)
    _, _, p1 = fmm.farfield(s, L=3, tree=tr, pair_tau=1.0, return_parts=True)
    tau = tau_in_gap(p1["norm2"], q)
    K, E, p = fmm.farfield(s, L=3, tree=tr, pair_tau=tau, return_parts=True)
    drop = ~p["keep"]
    assert drop.any() and p["keep"].any()
    assert np.array_equal(drop, drop.T)
    assert abs(E - (E0 - e[drop].sum())) <= 1e-12 * abs(E0)


def test_tau_above_all_norms_leaves_nothing(loc):
    s, tr, K0, E0, parts = loc
    _, _, p1 = fmm.farfield(s, L=3, tree=tr, pair_tau=1.0, return_parts=True)
    tau = 2.0 * float(np.sqrt(p1["norm2"].max()))
    K, E = fmm.farfield(s, L=3, tree=tr, pair_tau=tau)
    assert np.all(K == 0) and E == 0.0


def test_diagonal_pairs_survive(loc):
    s, tr, K0, E0, parts = loc
    nleaf = tr["nbox"] - tr["level_off"][tr["depth"]]
    tau = 0.99 / np.sqrt(nleaf)
    _, _, p = fmm.farfield(s, L=3, tree=tr, pair_tau=tau, return_parts=True)
    assert np.all(np.diag(p["keep"]))


def test_localised_orbitals_screen_well(loc):
    """Many pairs of localised orbitals on a line are negligible: dropping
    those below 1e-3 removes a quarter of them and changes the energy by far
    less than 1e-6 Eh."""
    s, tr, K0, E0, parts = loc
    K, E, p = fmm.farfield(s, L=3, tree=tr, pair_tau=1e-3, return_parts=True)
    assert p["keep"].mean() < 0.8
    assert abs(E - E0) < 1e-7


def test_cauchy_schwarz_pair_bound(loc):
    """The bound that lets step (a) skip whole tiles under screening:
    n_ij^2 <= sum_X a_iX^2 b_jX^2, a_iX^2 = sum_{r in S_X} C_ri^2,
    b_jX^2 = sum_{l, m} sum_{r in S_X} |O^{rj,X}_lm|^2 (Cauchy-Schwarz over
    the leaf's AO rows), for every pair, with O^{ij} from the (min, max)
    ordering as the screening uses it."""
    s, tr, K0, E0, parts = loc
    W = parts["W"]
    _, _, p = fmm.farfield(s, L=3, tree=tr, pair_tau=1.0, return_parts=True)
    a2 = np.array([np.sum(s.C[S] ** 2, axis=0) for S in tr["ao_sets"]])
    b2 = np.array([np.sum(np.abs(Wb) ** 2, axis=(0, 1)) for Wb in W])
    U = a2.T @ b2
    iu = np.triu_indices(s.nocc)
    assert np.all(p["norm2"][iu] <= U[iu] * (1 + 1e-12))
