"""Brute-force far-field exchange from exact ERIs (no multipole expansion).

    K^ff,exact_ri = 2 sum_j sum_{(A,B) far} sum_{(r,s) in A, (t,u) in B}
                    C_sj C_tj C_ui (rs|tu)

over kept shell pairs (r,s) owned by leaf A and (t,u) owned by leaf B, with A
and B not neighbours (Eq. occex restricted to the far field; the ERIs are
Eq. erib).  occ-FMM-K approximates exactly this sum; its error must fall with
the multipole rank.  Only for tiny systems.

Test infrastructure only (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np

from . import gauss


def far_eri_tensor(basis, tree):
    """G[r,s,t,u] = (rs|tu) if the shell pairs of (r,s) and (t,u) sit in
    non-neighbouring leaves, else 0."""
    shells = gauss.shell_data(basis)
    norms = gauss.contracted_norms(shells)
    aoff = basis.shell_ao_offset
    n = basis.nao
    key = tree["box_key"]
    leaf = tree["leaf_of_pair"]
    pa, pb = tree["pair_a"], tree["pair_b"]
    npair = len(pa)
    quartets, slots = [], []
    for x in range(npair):
        for y in range(npair):
            if np.max(np.abs(key[leaf[x]] - key[leaf[y]])) <= 1:
                continue
            quartets.append((int(pa[x]), int(pb[x]), int(pa[y]), int(pb[y])))
            slots.append((x, y))
    blocks = gauss.eri_quartets(shells, norms, quartets) if quartets else []
    G = np.zeros((n, n, n, n))
    for (a, b, c, d), blk in zip(quartets, blocks):
        ra = slice(aoff[a], aoff[a + 1])
        rb = slice(aoff[b], aoff[b + 1])
        rc = slice(aoff[c], aoff[c + 1])
        rd = slice(aoff[d], aoff[d + 1])
        # both orderings of each pair carry the same integral
        for (s1, s2, b1) in ((ra, rb, blk), (rb, ra, np.transpose(blk, (1, 0, 2, 3)))):
            G[s1, s2, rc, rd] = b1
            G[s1, s2, rd, rc] = np.transpose(b1, (0, 1, 3, 2))
    return G


def farfield_exact(basis, tree, C):
    G = far_eri_tensor(basis, tree)
    # (rj|ji) = sum_{s,t,u} C_sj C_tj C_ui (rs|tu)
    X = np.einsum("rstu,sj,tj->ruj", G, C, C)
    K = 2.0 * np.einsum("ruj,ui->ri", X, C)
    E = -0.5 * float(np.sum(C * K))
    return K, E
