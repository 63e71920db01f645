"""occ-FMM-K far-field exchange, complex FP64, step by step in the paper's order
(Sec. II, "The traditional FMM algorithm is modified as follows").

  0. AO-pair multipoles O^{rs,X}_lm about the centre X of the leaf that owns
     the pair (definition after Eq. eri; X unique to each pair).
  1. MO transforms (Eq. motrans):
        O^{rj,X}_lm = sum_s O^{rs,X}_lm C_sj,   O^{ij,X}_lm = sum_r O^{rj,X}_lm C_ri
  2. Occupied M2M, leaves up to level 2 (first of the occupied M2M/M2L/L2L
     equations, the per-(i,j) form of Eq. fmm1).
  3. Occupied M2L over each interaction list, levels 2..D (Eq. fmmex / fmm2).
  4. Occupied L2L, level 2 down to the leaves (Eq. fmm3, M read as the local
     expansion Mcal).
  5. K^ff_ri = 2 sum_j sum_lm O^{rj,X}_lm Mcal^{ij}_lm(X) summed over the leaf
     boxes X (Eq. kri with the factor 2 of Eq. occex; see below), and
     E^ff_x = -1/2 sum_ri C_ri K^ff_ri = -sum_ij (ij|ji)^ff.

Readings (the paper is silent or inconsistent):
* Eq. kri omits the factor 2 of Eq. occex; K_ri = 2 sum_j (rj|ji) is used.
* A pair (r, s) assigned to box X contributes to O^{rj,X} and, through the
  symmetric ordering, to O^{sj,X}.
* Per-edge truncation (``lmax_edges``): the M2L operator of an edge keeps only
  output and input ranks <= L_e; M2M and L2L keep the full L.

Occupied-pair screening (``pair_tau``; the paper's proposed extension to
localised orbitals, Sec. IV): after step 1 a pair (i, j) whose pair-density
multipoles are negligible over all leaves,
    n_ij^2 = sum_X sum_{l, m=-l..l} |O^{ij,X}_lm|^2 < tau^2,
is dropped: its multipoles are set to zero before step 2, so it has no local
expansion and no part in K.  Pairs are independent in steps 2-5, so the
energy changes by exactly the dropped pairs' own contributions
e_ij = -sum_X sum_lm O^{ij,X}_lm Mcal^{ij}_lm(X).

Everything runs for a subset I of occupied columns i when ``i_subset`` is
given: K_{r,i in I} needs O^{ij}, Mcal^{ij} for i in I and all j only, so the
result is exact for those columns.

Test infrastructure only (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np

from . import gauss, solid
from .tree import build_tree


def pair_multipoles(basis, tree, L):
    """Step 0: per kept shell pair, complex [na, nb, (L+1)^2] about its leaf centre."""
    pairs = list(zip(tree["pair_a"].tolist(), tree["pair_b"].tolist()))
    X = tree["centre"][tree["leaf_of_pair"]]
    return gauss.ao_pair_multipoles(basis, pairs, X, L)


def half_transform(basis, tree, Opair, C, L):
    """Step 1a: W[leaf] = O^{rj,X}_lm as [nlm, |S_B|, nocc] on each leaf's AO set."""
    D = tree["depth"]
    lo = tree["level_off"][D]
    aoff = basis.shell_ao_offset
    nocc = C.shape[1]
    nlm = solid.nlm(L)
    W = []
    pos = []
    for S in tree["ao_sets"]:
        W.append(np.zeros((nlm, len(S), nocc), dtype=np.complex128))
        pos.append({int(r): k for k, r in enumerate(S)})
    for k, (a, b) in enumerate(zip(tree["pair_a"].tolist(), tree["pair_b"].tolist())):
        leaf = tree["leaf_of_pair"][k] - lo
        O = Opair[k]                                  # [na, nb, nlm]
        ra = range(aoff[a], aoff[a + 1])
        rb = range(aoff[b], aoff[b + 1])
        for ia, r in enumerate(ra):
            for ib, s in enumerate(rb):
                # (r, s): O^{rs} C_sj into row r
                W[leaf][:, pos[leaf][r], :] += O[ia, ib, :, None] * C[s][None, :]
                if a != b:
                    # (s, r): the same pair in the other order, O^{sr} = O^{rs}
                    W[leaf][:, pos[leaf][s], :] += O[ia, ib, :, None] * C[r][None, :]
    return W


def full_transform(tree, W, C, i_cols):
    """Step 1b: O^{ij,X}_lm = sum_r O^{rj,X}_lm C_ri, as [nlm, |I|, nocc] per leaf."""
    out = []
    for S, Wb in zip(tree["ao_sets"], W):
        Cs = C[S][:, i_cols]                           # [|S_B|, |I|]
        out.append(np.einsum("ri,lrj->lij", Cs, Wb))
    return out


def farfield(system_or_basis, C=None, L=None, tree=None, i_subset=None,
             lmax_edges=None, pair_thresh=1e-14, return_parts=False, Opair=None, W=None,
             pair_tau=None):
    """Far-field K^ff (n_AO x |I|) and E^ff for the columns in ``i_subset``.

    ``Opair`` / ``W`` may carry step 0 and the first half of step 1 from an
    earlier call on the same tree, rank and C (they do not depend on I)."""
    if hasattr(system_or_basis, "basis"):
        sysm = system_or_basis
        basis, C = sysm.basis, sysm.C if C is None else C
        L = sysm.lmax if L is None else L
        if tree is None:
            tree = build_tree(basis, sysm.depth, sysm.target_atoms_per_leaf, pair_thresh)
    else:
        basis = system_or_basis
        if tree is None:
            raise ValueError("tree required")
    nocc = C.shape[1]
    i_cols = np.arange(nocc) if i_subset is None else np.asarray(i_subset)
    nI = len(i_cols)
    nlm = solid.nlm(L)
    D = tree["depth"]
    nbox = tree["nbox"]
    lo_leaf = tree["level_off"][D]

    if Opair is None:
        Opair = pair_multipoles(basis, tree, L)
    if W is None:
        W = half_transform(basis, tree, Opair, C, L)
    Oleaf = full_transform(tree, W, C, i_cols)
    # occupied-pair screening: drop pairs with negligible multipoles on every leaf
    # (the norm of an unordered pair is taken from O^{ab}, a = min(i, j),
    # b = max(i, j), so that (i, j) and (j, i) share one decision)
    keep = None
    norm2 = None
    if pair_tau is not None and pair_tau > 0:
        norm2 = np.zeros((nI, nocc))
        upper = i_cols[:, None] <= np.arange(nocc)[None, :]
        for S, Wb, Ob in zip(tree["ao_sets"], W, Oleaf):
            Ot = np.einsum("rj,lri->lij", C[S], Wb[:, :, i_cols])      # O^{ji} for i in I
            norm2 += np.sum(np.abs(np.where(upper[None], Ob, Ot)) ** 2, axis=0)
        keep = norm2 >= pair_tau ** 2
        Oleaf = [Ob * keep[None] for Ob in Oleaf]

    # multipoles O^{ij} of every box, [nbox, nlm, |I|, nocc]
    Obox = np.zeros((nbox, nlm, nI, nocc), dtype=np.complex128)
    for k, Ob in enumerate(Oleaf):
        Obox[lo_leaf + k] = Ob
    # Step 2: M2M from level D up to level 2
    for lev in range(D, 2, -1):
        for c in range(tree["level_off"][lev], tree["level_off"][lev + 1]):
            p = tree["parent"][c]
            T = solid.m2m_matrix(tree["centre"][c] - tree["centre"][p], L)
            Obox[p] += np.einsum("ab,bij->aij", T, Obox[c])
    # Step 3: M2L over interaction lists
    Mbox = np.zeros_like(Obox)
    nedge = len(tree["m2l_tgt"])
    for e in range(nedge):
        t = tree["m2l_tgt"][e]
        s = tree["m2l_src"][e]
        Le = L if lmax_edges is None else int(lmax_edges[e])
        T = solid.m2l_matrix(tree["centre"][t] - tree["centre"][s], L, Lout=Le, Lin=Le)
        Mbox[t] += np.einsum("ab,bij->aij", T, Obox[s])
    # Step 4: L2L from level 2 down to D
    for lev in range(3, D + 1):
        for c in range(tree["level_off"][lev], tree["level_off"][lev + 1]):
            p = tree["parent"][c]
            T = solid.l2l_matrix(tree["centre"][c] - tree["centre"][p], L)
            Mbox[c] += np.einsum("ab,bij->aij", T, Mbox[p])
    # Step 5: K^ff_ri = 2 sum_X sum_j sum_lm O^{rj,X}_lm Mcal^{ij}_lm(X)
    K = np.zeros((basis.nao, nI), dtype=np.complex128)
    for k, (S, Wb) in enumerate(zip(tree["ao_sets"], W)):
        Ml = Mbox[lo_leaf + k]                          # [nlm, |I|, nocc]
        K[S] += 2.0 * np.einsum("lrj,lij->ri", Wb, Ml)
    if np.max(np.abs(K.imag)) > 1e-9 * max(1.0, np.max(np.abs(K.real))):
        raise AssertionError("far-field K has a non-negligible imaginary part")
    K = K.real
    E = -0.5 * float(np.sum(C[:, i_cols] * K))
    if return_parts:
        return K, E, dict(tree=tree, W=W, Obox=Obox, Mbox=Mbox, Opair=Opair, keep=keep, norm2=norm2)
    return K, E


def edge_energies(tree, Obox, L, lmax_list):
    """Energy contribution of every M2L edge at each truncation rank.

    The translations M2M and L2L are exact re-expansions, so the far-field
    energy splits over M2L edges:  E = -sum_edges sum_ij sum_lm
    O^{ji}_lm(B) [T_{B<-B'} O^{ij}(B')]_lm.  Returns [nedge, len(lmax_list)]
    (requires Obox over all i)."""
    nedge = len(tree["m2l_tgt"])
    out = np.zeros((nedge, len(lmax_list)))
    for e in range(nedge):
        t = tree["m2l_tgt"][e]
        s = tree["m2l_src"][e]
        R = tree["centre"][t] - tree["centre"][s]
        for q, Le in enumerate(lmax_list):
            T = solid.m2l_matrix(R, L, Lout=Le, Lin=Le)
            Mts = np.einsum("ab,bij->aij", T, Obox[s])
            out[e, q] = -float(np.real(np.einsum("aji,aij->", Obox[t], Mts)))
    return out
