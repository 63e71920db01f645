"""Far-field Coulomb matrix by the FMM, complex FP64, in the paper's steps
(Sec. II, from "When constructing the Coulomb matrix" to the J^ff formula):

  0. AO-pair multipoles O^{tu,X'}_lm about the centre of the leaf owning the
     pair (the same integrals as for exchange).
  1. Density multipoles of every leaf: O^{X'}_lm = sum_{tu in X'} D_tu O^{tu,X'}_lm
     (both orderings of a pair t != u).
  2. M2M from the leaves up to level 2 (Eq. fmm1), M2L over the interaction
     lists (Eq. fmmc / fmm2), L2L down to the leaves (Eq. fmm3).
  3. J^ff_rs = sum_lm O^{rs,X}_lm Mcal_lm(X) for every kept pair (r, s) of leaf
     X, and E_J^ff = 1/2 sum_rs D_rs J^ff_rs.

D is the (symmetric) density matrix, for closed shells D = 2 C C^T.

Test infrastructure only (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np

from . import solid
from .fmm import pair_multipoles


def farfield_J(basis, D, L, tree, Opair=None):
    """J^ff [nao, nao] (zero outside kept pairs) and E_J^ff."""
    nlm = solid.nlm(L)
    depth = tree["depth"]
    nbox = tree["nbox"]
    aoff = basis.shell_ao_offset
    if Opair is None:
        Opair = pair_multipoles(basis, tree, L)
    pairs = list(zip(tree["pair_a"].tolist(), tree["pair_b"].tolist()))
    # Step 1: density multipoles of the leaves
    Obox = np.zeros((nbox, nlm), dtype=np.complex128)
    for k, (a, b) in enumerate(pairs):
        X = tree["leaf_of_pair"][k]
        O = Opair[k]
        for ia, r in enumerate(range(aoff[a], aoff[a + 1])):
            for ib, s in enumerate(range(aoff[b], aoff[b + 1])):
                Obox[X] += D[r, s] * O[ia, ib]
                if a != b:
                    Obox[X] += D[s, r] * O[ia, ib]
    # Step 2: M2M, M2L, L2L on the one density channel
    for lev in range(depth, 2, -1):
        for c in range(tree["level_off"][lev], tree["level_off"][lev + 1]):
            p = tree["parent"][c]
            Obox[p] += solid.m2m_matrix(tree["centre"][c] - tree["centre"][p], L) @ Obox[c]
    Mbox = np.zeros_like(Obox)
    for t, s in zip(tree["m2l_tgt"].tolist(), tree["m2l_src"].tolist()):
        Mbox[t] += solid.m2l_matrix(tree["centre"][t] - tree["centre"][s], L) @ Obox[s]
    for lev in range(3, depth + 1):
        for c in range(tree["level_off"][lev], tree["level_off"][lev + 1]):
            p = tree["parent"][c]
            Mbox[c] += solid.l2l_matrix(tree["centre"][c] - tree["centre"][p], L) @ Mbox[p]
    # Step 3: J^ff on the kept pairs
    J = np.zeros((basis.nao, basis.nao), dtype=np.complex128)
    for k, (a, b) in enumerate(pairs):
        X = tree["leaf_of_pair"][k]
        O = Opair[k]
        for ia, r in enumerate(range(aoff[a], aoff[a + 1])):
            for ib, s in enumerate(range(aoff[b], aoff[b + 1])):
                v = np.sum(O[ia, ib] * Mbox[X])
                J[r, s] = v
                J[s, r] = v
    if np.max(np.abs(J.imag)) > 1e-9 * max(1.0, np.max(np.abs(J.real))):
        raise AssertionError("far-field J has a non-negligible imaginary part")
    J = J.real
    return J, 0.5 * float(np.sum(D * J))


def farfield_J_exact(basis, tree, D):
    """The same far field from exact four-centre integrals over far boxes:
    J_rs = sum_tu (rs|tu) D_tu over pairs in non-neighbouring leaves."""
    from .brute import far_eri_tensor
    G = far_eri_tensor(basis, tree)
    J = np.einsum("rstu,tu->rs", G, D)
    return J, 0.5 * float(np.sum(D * J))
