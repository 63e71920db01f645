"""Box hierarchy for the far field (Sec. II, the paragraphs on the box
hierarchy, interaction lists and FMM parameters).

Readings of the paper used here (the paper defers the details to references):
* Every kept shell pair (a <= b) is assigned, as a whole, to the leaf box that
  contains its centre, the weight-averaged Gaussian product centre
  sum_pq w_pq P_pq / sum_pq w_pq with w_pq = exp(-mu_pq |A-B|^2).  "X is unique
  to each pair r, s" (Sec. II) -- so a pair is never split across boxes.
* Shell-pair screen: keep (a, b) if max over primitive pairs of
  |c_p c_q| (2 sqrt(a_p a_q)/(a_p + a_q))^(3/2) exp(-mu |A-B|^2) > thresh
  (the overlap of the two normalised primitives, times the coefficients).
* Root cube: min corner = min over pair centres - delta, side = largest
  extent + 2 delta, delta = 1e-6 * largest extent.  Depth D = number of
  subdivisions; leaf boxes have side/2^D.  Leaf index = floor((x - x0)/h_D),
  clamped to [0, 2^D - 1]; coarser indices are leaf indices shifted right.
* depth = 0 chooses D in 1..12 minimising |natom / (non-empty leaves by atom
  position) - target|, ties to the smaller D.
* Only non-empty boxes exist.  Boxes are ordered by (level, ix, iy, iz).
* Neighbours: Chebyshev distance <= 1 at the same level.  The interaction
  list of B (levels >= 2) holds the boxes whose parent is the parent of B or
  one of its neighbours, and that are not neighbours of B ("well separated"
  = nearest-neighbour boxes excluded).

Test infrastructure only (see oracle/__init__.py).
"""
from __future__ import annotations

import math

import numpy as np


# The C library's exp: pair centres are compared bit for bit with the host
# implementation, and a centre that lies exactly on a box face (the middle of
# a symmetric molecule) must round the same way on both sides.
_exp = np.frompyfunc(math.exp, 1, 1)


def _exp_f64(x):
    return _exp(x).astype(np.float64)


def shell_pairs(basis, thresh: float = 1e-14):
    """Screened shell pairs (a <= b) and their centres, in (a, b) order."""
    poff = basis.shell_prim_offset
    xyz = basis.xyz
    ns = basis.nshell
    a_idx, b_idx = np.triu_indices(ns)
    A = xyz[basis.shell_atom[a_idx]]
    B = xyz[basis.shell_atom[b_idx]]
    R2 = np.sum((A - B) ** 2, axis=1)
    npmax = int(basis.shell_nprim.max())
    est = np.zeros(len(a_idx))
    sw = np.zeros(len(a_idx))
    swx = np.zeros((len(a_idx), 3))
    na = basis.shell_nprim[a_idx]
    nb = basis.shell_nprim[b_idx]
    for p in range(npmax):
        for q in range(npmax):
            ok = (p < na) & (q < nb)
            ia = poff[a_idx] + np.minimum(p, na - 1)
            ib = poff[b_idx] + np.minimum(q, nb - 1)
            ea = basis.exps[ia]
            eb = basis.exps[ib]
            ca = basis.coefs[ia]
            cb = basis.coefs[ib]
            pp = ea + eb
            mu = ea * eb / pp
            w = _exp_f64(-mu * R2)
            t = 2.0 * np.sqrt(ea * eb) / pp
            e = np.abs(ca * cb) * (t * np.sqrt(t)) * w
            est = np.where(ok, np.maximum(est, e), est)
            sw = np.where(ok, sw + w, sw)
            P = (ea[:, None] * A + eb[:, None] * B) / pp[:, None]
            swx = np.where(ok[:, None], swx + w[:, None] * P, swx)
    keep = est > thresh
    centres = swx[keep] / sw[keep][:, None]
    return a_idx[keep].astype(np.int64), b_idx[keep].astype(np.int64), centres


def _keys(x, x0, h, n):
    k = np.floor((x - x0) / h).astype(np.int64)
    return np.clip(k, 0, n - 1)


def build_tree(basis, depth: int = 0, target_atoms_per_leaf: float = 8.0,
               pair_thresh: float = 1e-14):
    sa, sb, cen = shell_pairs(basis, pair_thresh)
    lo = cen.min(axis=0)
    hi = cen.max(axis=0)
    extent = float(np.max(hi - lo))
    delta = 1e-6 * extent if extent > 0 else 1e-6
    x0 = lo - delta
    side = extent + 2.0 * delta
    if depth <= 0:
        best = None
        for D in range(1, 13):
            n = 1 << D
            h = side / n
            ka = _keys(basis.xyz, x0, h, n)
            occupied = len({tuple(k) for k in ka.tolist()})
            mean = basis.natom / occupied
            err = abs(mean - target_atoms_per_leaf)
            if best is None or err < best[0]:
                best = (err, D)
        depth = best[1]
    D = depth
    nD = 1 << D
    hD = side / nD
    leafkey = _keys(cen, x0, hD, nD)

    # boxes per level, ordered (level, ix, iy, iz)
    levels = []
    for lev in range(D + 1):
        kk = leafkey >> (D - lev)
        uniq = sorted({tuple(k) for k in kk.tolist()})
        levels.append(uniq)
    box_level, box_key, level_off = [], [], [0]
    index = {}
    for lev, uniq in enumerate(levels):
        for k in uniq:
            index[(lev,) + k] = len(box_level)
            box_level.append(lev)
            box_key.append(k)
        level_off.append(len(box_level))
    box_key = np.array(box_key, dtype=np.int64).reshape(-1, 3)
    box_level = np.array(box_level, dtype=np.int64)
    parent = np.full(len(box_level), -1, dtype=np.int64)
    for b in range(len(box_level)):
        lev = box_level[b]
        if lev > 0:
            parent[b] = index[(lev - 1,) + tuple((box_key[b] >> 1).tolist())]
    h = np.array([side / (1 << lev) for lev in range(D + 1)])
    centre = np.zeros((len(box_level), 3))
    for b in range(len(box_level)):
        lev = box_level[b]
        centre[b] = x0 + (box_key[b] + 0.5) * h[lev]

    # interaction lists, levels 2..D, sorted by (target, source)
    m2l_t, m2l_s = [], []
    for lev in range(2, D + 1):
        ids = list(range(level_off[lev], level_off[lev + 1]))
        keys = box_key[ids]
        pk = keys >> 1
        for a, b in enumerate(ids):
            dpar = np.max(np.abs(pk - pk[a]), axis=1)
            dself = np.max(np.abs(keys - keys[a]), axis=1)
            for c in np.nonzero((dpar <= 1) & (dself > 1))[0]:
                m2l_t.append(b)
                m2l_s.append(ids[c])

    leaf_of_pair = np.array([index[(D,) + tuple(k)] for k in leafkey.tolist()], dtype=np.int64)

    # AO sets of each leaf
    aoff = basis.shell_ao_offset
    nleaf = level_off[D + 1] - level_off[D]
    ao_sets = [set() for _ in range(nleaf)]
    for a, b, L in zip(sa.tolist(), sb.tolist(), leaf_of_pair.tolist()):
        s = ao_sets[L - level_off[D]]
        s.update(range(aoff[a], aoff[a + 1]))
        s.update(range(aoff[b], aoff[b + 1]))
    ao_sets = [np.array(sorted(s), dtype=np.int64) for s in ao_sets]

    return dict(depth=D, x0=x0, side=side, h=h, nbox=len(box_level),
                level_off=np.array(level_off, dtype=np.int64), box_level=box_level,
                box_key=box_key, parent=parent, centre=centre,
                m2l_tgt=np.array(m2l_t, dtype=np.int64), m2l_src=np.array(m2l_s, dtype=np.int64),
                pair_a=sa, pair_b=sb, pair_centre=cen, leaf_of_pair=leaf_of_pair,
                ao_sets=ao_sets)


def neighbours(tree, b):
    lev = tree["box_level"][b]
    lo, hi = tree["level_off"][lev], tree["level_off"][lev + 1]
    keys = tree["box_key"][lo:hi]
    d = np.max(np.abs(keys - tree["box_key"][b]), axis=1)
    return [lo + i for i in np.nonzero(d <= 1)[0]]
