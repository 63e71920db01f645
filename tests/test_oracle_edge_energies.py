"""Pins for the oracle's per-edge energy split (the learned selector's labels).

M2M and L2L re-expand exactly, so the far-field energy is a sum over M2L
edges of bilinear forms in the occupied multipoles of the edge's two boxes
(Sec. II, the occupied M2L of Eq. fmmex followed by Eq. kri).  Two facts fix
``fmm.edge_energies`` without reference to its own code:

* summed over the edges at one truncation rank k, it is the far-field energy
  of the whole method run at rank k (truncating an M2L operator to output and
  input ranks <= k is the rank-k method: M2M output of rank l depends only on
  input ranks <= l, and L2L output of rank l only on input ranks >= l);
* with a rank r_e per edge, the sum of each edge's entry at r_e is the energy
  of the method run with those per-edge ranks (``lmax_edges``).

A dropped term, a sign error or a wrong box in the bilinear form fails both.
"""
import numpy as np
import pytest

from oracle import fmm
from oracle import tree as otree
from paper_1708_05353_gb300 import inputs


def _setup(s, L, depth):
    tr = otree.build_tree(s.basis, depth, s.target_atoms_per_leaf)
    _, E, parts = fmm.farfield(s, L=L, tree=tr, return_parts=True)
    return tr, E, parts


def _rank(s, tr, parts, k, **kw):
    """The method at rank k, reusing the rank-L pair multipoles and half
    transform (their components of rank <= k are the rank-k ones)."""
    nk = (k + 1) ** 2
    return fmm.farfield(s, L=k, tree=tr, Opair=[o[..., :nk] for o in parts["Opair"]],
                        W=[w[:nk] for w in parts["W"]], **kw)


@pytest.fixture(scope="module")
def sp():
    s = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    L = 5
    tr, E, parts = _setup(s, L, 3)
    return s, L, tr, E, parts


@pytest.fixture(scope="module")
def water():
    s = inputs.water(nmol=6, lmax=3)
    L = 3
    tr, E, parts = _setup(s, L, 2)
    return s, L, tr, E, parts


@pytest.mark.parametrize("which", ["sp", "water"])
def test_edge_sum_is_method_energy_at_each_rank(which, sp, water):
    s, L, tr, E, parts = {"sp": sp, "water": water}[which]
    assert len(tr["m2l_tgt"]) > 0
    ranks = list(range(L + 1))
    ee = fmm.edge_energies(tr, parts["Obox"], L, ranks)
    assert ee.shape == (len(tr["m2l_tgt"]), L + 1)
    assert abs(ee[:, L].sum() - E) <= 1e-12 * abs(E)
    for k in ranks[:-1]:
        _, Ek = _rank(s, tr, parts, k)
        assert abs(ee[:, k].sum() - Ek) <= 1e-12 * abs(Ek), (k, ee[:, k].sum(), Ek)


@pytest.mark.parametrize("which", ["sp", "water"])
def test_edge_sum_with_per_edge_ranks(which, sp, water):
    s, L, tr, E, parts = {"sp": sp, "water": water}[which]
    ne = len(tr["m2l_tgt"])
    ee = fmm.edge_energies(tr, parts["Obox"], L, list(range(L + 1)))
    for seed in (1, 2):
        r = np.random.default_rng(seed).integers(0, L + 1, size=ne)
        _, Er = _rank(s, tr, parts, L, lmax_edges=r)
        got = float(ee[np.arange(ne), r].sum())
        assert abs(got - Er) <= 1e-12 * abs(Er), (seed, got, Er)


def test_edge_energy_sign_and_order(sp):
    """One edge's label difference between ranks L and 0 is exactly the
    energy change of the method when only that edge is cut to rank 0."""
    s, L, tr, E, parts = sp
    Obox = parts["Obox"]
    ne = len(tr["m2l_tgt"])
    ee = fmm.edge_energies(tr, Obox, L, [L])[:, 0]
    # rank 0 keeps only the monopole-monopole term; the difference between
    # rank L and rank 0 on one edge is that edge's higher-order part
    e0 = fmm.edge_energies(tr, Obox, L, [0])[:, 0]
    k = int(np.argmax(np.abs(ee - e0)))
    r = np.full(ne, L)
    r[k] = 0
    _, Er = _rank(s, tr, parts, L, lmax_edges=r)
    assert abs((E - Er) - (ee[k] - e0[k])) <= 1e-12 * abs(E)
