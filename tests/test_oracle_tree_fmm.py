"""Pins for the oracle's box hierarchy and its occ-FMM-K far field.

* Tree: every pair centre lies in its leaf box; interaction lists exclude
  neighbours; and every ordered pair of distinct leaves is either neighbouring
  or covered by exactly one M2L edge between their ancestors (the far field is
  partitioned exactly once, Sec. II).
* Far field: converges with the multipole rank to the brute-force far-field
  exchange built from exact ERIs (Eq. occex over far pairs, Eq. erib), for
  s-only and s/p systems.
* L = 0 reduces to a closed form in overlaps over box-centre distances.
* Symmetries: O^{ij} = O^{ji}, Mcal^{ij} = Mcal^{ji}, the MO block K_ij is
  symmetric, the monopole sum rule sum_X O^{ij,X}_00 = delta_ij, invariance
  under rigid shifts and under a cyclic permutation of the axes.
"""
import numpy as np
import pytest

from oracle import brute, fmm, solid
from oracle import tree as otree
from paper_1708_05353_gb300 import inputs


@pytest.fixture(scope="module")
def line():
    s = inputs.tiny_line()
    tr = otree.build_tree(s.basis, s.depth, 8.0)
    return s, tr


@pytest.fixture(scope="module")
def sp():
    s = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    tr = otree.build_tree(s.basis, s.depth, 8.0)
    return s, tr


def test_tree_shape_line(line):
    s, tr = line
    assert tr["depth"] == 3
    np.testing.assert_array_equal(tr["level_off"], [0, 1, 3, 7, 15])
    assert len(tr["m2l_tgt"]) == 24


def _check_tree(tr):
    D = tr["depth"]
    lo = tr["level_off"]
    h = tr["h"]
    # pair centre inside its leaf (half-open box, clamped at the top face)
    for c, leaf in zip(tr["pair_centre"], tr["leaf_of_pair"]):
        k = tr["box_key"][leaf]
        x = (c - tr["x0"]) / h[D]
        assert np.all(x >= k - 1e-12) and np.all(x <= k + 1 + 1e-12)
    # interaction lists: same level, not neighbours, parents neighbours
    key = tr["box_key"]
    for t, s_ in zip(tr["m2l_tgt"], tr["m2l_src"]):
        assert tr["box_level"][t] == tr["box_level"][s_]
        assert np.max(np.abs(key[t] - key[s_])) > 1
        assert np.max(np.abs(key[tr["parent"][t]] - key[tr["parent"][s_]])) <= 1
    # exact partition of the far field over leaf pairs
    edges = set(zip(tr["m2l_tgt"].tolist(), tr["m2l_src"].tolist()))
    leaves = range(lo[D], lo[D + 1])

    def ancestors(b):
        out = [b]
        while tr["parent"][out[-1]] >= 0:
            out.append(tr["parent"][out[-1]])
        return out
    for A in leaves:
        anc_a = ancestors(A)
        for B in leaves:
            if A == B:
                continue
            anc_b = ancestors(B)
            cover = sum((x, y) in edges for x, y in zip(anc_a, anc_b))
            near = np.max(np.abs(key[A] - key[B])) <= 1
            assert cover == (0 if near else 1)


def test_tree_invariants(line, sp):
    _check_tree(line[1])
    _check_tree(sp[1])


def test_tree_invariants_3d():
    s = inputs.water(nmol=12, lmax=2)
    tr = otree.build_tree(s.basis, 2, 8.0)
    _check_tree(tr)


def test_far_field_converges_to_brute_force_s(line):
    s, tr = line
    Kx, Ex = brute.farfield_exact(s.basis, tr, s.C)
    errs = []
    for L in (2, 6, 10):
        K, E = fmm.farfield(s, L=L, tree=tr)
        errs.append(abs(E - Ex))
        assert np.max(np.abs(K - Kx)) < 0.1 * np.max(np.abs(Kx))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 3e-5 * abs(Ex)


def test_far_field_converges_to_brute_force_sp(sp):
    s, tr = sp
    assert len(tr["m2l_tgt"]) > 0
    Kx, Ex = brute.farfield_exact(s.basis, tr, s.C)
    errs = []
    kerr = []
    for L in (1, 3, 6, 9):
        K, E = fmm.farfield(s, L=L, tree=tr)
        errs.append(abs(E - Ex))
        kerr.append(np.max(np.abs(K - Kx)))
    assert kerr[0] > kerr[1] > kerr[2] > kerr[3]
    assert kerr[3] < 1e-3 * np.max(np.abs(Kx))
    assert errs[3] < 1e-3 * abs(Ex)


def test_L0_closed_form(line):
    """At L = 0 every translation moves only monopoles, so
    K_ri = 2 sum_edges sum_j (P_A C)_rj (C^T P_A' C)_ij / |X_B - X_B'|
    with P_A the overlap restricted to pairs owned by leaves A under B."""
    s, tr = line
    S = inputs.overlap_matrix(s.basis)
    C = s.C
    aoff = s.basis.shell_ao_offset
    D = tr["depth"]
    lo = tr["level_off"]
    n = s.basis.nao
    Pleaf = {b: np.zeros((n, n)) for b in range(lo[D], lo[D + 1])}
    for a, b, leaf in zip(tr["pair_a"], tr["pair_b"], tr["leaf_of_pair"]):
        ra = slice(aoff[a], aoff[a + 1])
        rb = slice(aoff[b], aoff[b + 1])
        Pleaf[leaf][ra, rb] = S[ra, rb]
        Pleaf[leaf][rb, ra] = S[rb, ra]

    def under(B):
        out = []
        for leaf in Pleaf:
            x = leaf
            while x >= 0 and x != B:
                x = tr["parent"][x]
            if x == B:
                out.append(leaf)
        return out
    K = np.zeros((n, C.shape[1]))
    for t, src in zip(tr["m2l_tgt"], tr["m2l_src"]):
        Pt = sum(Pleaf[x] for x in under(t))
        Ps = sum(Pleaf[x] for x in under(src))
        R = np.linalg.norm(tr["centre"][t] - tr["centre"][src])
        K += 2.0 * (Pt @ C) @ (C.T @ Ps @ C).T / R
    Kf, Ef = fmm.farfield(s, L=0, tree=tr)
    np.testing.assert_allclose(Kf, K, rtol=1e-10, atol=1e-13)


def test_symmetries_and_sum_rule(sp):
    s, tr = sp
    K, E, parts = fmm.farfield(s, L=3, tree=tr, return_parts=True)
    Ob, Mb = parts["Obox"], parts["Mbox"]
    np.testing.assert_allclose(Ob, np.swapaxes(Ob, 2, 3), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(Mb, np.swapaxes(Mb, 2, 3), rtol=1e-10, atol=1e-13)
    KMO = s.C.T @ K
    np.testing.assert_allclose(KMO, KMO.T, rtol=1e-9, atol=1e-12)
    D = tr["depth"]
    lo = tr["level_off"]
    mono = sum(Ob[b, solid.idx(0, 0)] for b in range(lo[D], lo[D + 1]))
    np.testing.assert_allclose(mono.real, np.eye(s.nocc), atol=1e-10)
    assert abs(E - (-0.5 * np.sum(s.C * K))) < 1e-15 + 1e-13 * abs(E)


def test_column_subset_is_exact(sp):
    s, tr = sp
    K, E = fmm.farfield(s, L=3, tree=tr)
    I = [3, 1]
    Ks, Es = fmm.farfield(s, L=3, tree=tr, i_subset=I)
    np.testing.assert_allclose(Ks, K[:, I], rtol=1e-12, atol=1e-15)


def _permute_axes(sysm, perm):
    """New coordinate k = old coordinate perm[k]; p rows of C follow."""
    b = sysm.basis
    nb = inputs.Basis(xyz=b.xyz[:, perm].copy(), elements=b.elements, shell_atom=b.shell_atom,
                      shell_l=b.shell_l, shell_nprim=b.shell_nprim, exps=b.exps, coefs=b.coefs)
    rows = []
    aoff = b.shell_ao_offset
    for sh in range(b.nshell):
        if b.shell_l[sh] == 0:
            rows.append(aoff[sh])
        else:
            rows.extend(aoff[sh] + np.array(perm))
    rows = np.array(rows)
    return inputs.System(sysm.name, nb, sysm.nocc, sysm.C[rows], sysm.depth,
                         sysm.target_atoms_per_leaf, sysm.lmax), rows


def test_axis_permutation_invariance():
    s = inputs.small_sp(natom=5, nocc=3, spacing=3.0, depth=3)
    s.basis.xyz[:, 1] += np.linspace(0, 4.0, 5)   # break the line's symmetry
    K, E = fmm.farfield(s, L=4)
    s2, rows = _permute_axes(s, [2, 0, 1])
    K2, E2 = fmm.farfield(s2, L=4)
    assert E2 == pytest.approx(E, rel=1e-11)
    np.testing.assert_allclose(K2, K[rows], rtol=1e-9, atol=1e-12)


def test_rigid_shift_invariance():
    # irregular spacing: a centre exactly on a box face (the middle of a
    # symmetric system) may change box under rounding after a shift
    s = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    s.basis.xyz[:, 0] += np.array([0.0, 0.11, -0.07, 0.05, 0.13, -0.02])
    K, E = fmm.farfield(s, L=3)
    b = s.basis
    nb = inputs.Basis(xyz=b.xyz + np.array([10.25, -3.5, 7.0]), elements=b.elements,
                      shell_atom=b.shell_atom, shell_l=b.shell_l, shell_nprim=b.shell_nprim,
                      exps=b.exps, coefs=b.coefs)
    s2 = inputs.System(s.name, nb, s.nocc, s.C, s.depth, 8.0, s.lmax)
    K2, E2 = fmm.farfield(s2, L=3)
    assert E2 == pytest.approx(E, rel=1e-10)
    np.testing.assert_allclose(K2, K, rtol=1e-8, atol=1e-12)
