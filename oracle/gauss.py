"""s/p Cartesian Gaussians: normalisation, AO-pair multipole integrals, Boys
function and McMurchie-Davidson electron-repulsion integrals.

* AO-pair multipole integrals (Sec. II, definition after Eq. eri):
      O^{rs,X}_lm = int phi_r(r) O_lm(r - X) phi_s(r) dr
  evaluated by tensor-product Gauss-Hermite quadrature about each primitive
  product centre.  The integrand is a polynomial of degree <= l + 2 per axis
  times a Gaussian, so n = L//2 + 2 nodes per axis integrate it exactly.
* ERIs (Eq. erib), (rs|tu) = int int phi_r phi_s (1) 1/r12 phi_t phi_u (2),
  by McMurchie-Davidson Hermite expansion, used only by the brute-force
  far-field reference.

Primitive normalisation: s: (2a/pi)^(3/4), p: (2a/pi)^(3/4) * 2 sqrt(a).
Contracted functions are renormalised to unit self-overlap.

Test infrastructure only (see oracle/__init__.py).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from . import solid


# ---------------------------------------------------------------------------
# AO bookkeeping
# ---------------------------------------------------------------------------

def shell_data(basis):
    """Per shell: centre, l, exponents, coefficients on normalised primitives
    multiplied by the primitive normalisation, AO offset."""
    poff = basis.shell_prim_offset
    aoff = basis.shell_ao_offset
    out = []
    for s in range(basis.nshell):
        e = basis.exps[poff[s]:poff[s + 1]].copy()
        c = basis.coefs[poff[s]:poff[s + 1]].copy()
        n = (2.0 * e / math.pi) ** 0.75
        if basis.shell_l[s] == 1:
            n = n * 2.0 * np.sqrt(e)
        out.append(dict(A=basis.xyz[basis.shell_atom[s]].copy(), l=int(basis.shell_l[s]),
                        e=e, c=c * n, ao=int(aoff[s]), nao=1 if basis.shell_l[s] == 0 else 3))
    return out


def _gh(n):
    x, w = np.polynomial.hermite.hermgauss(n)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel()
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1), W


def _cart_factor(pts, A, l):
    """Cartesian prefactor of the AO: 1 (s) or (r - A)_k (p, k = x, y, z)."""
    if l == 0:
        return np.ones(pts.shape[:-1] + (1,))
    return pts - A[..., None, :]


def pair_multipoles_raw(sa, sb, X, L, nquad=None):
    """Unnormalised multipole integrals of the contracted shell pair (sa, sb)
    about centres X.

    sa, sb: lists (one entry per pair) of shell dicts with the same l and the
    same number of primitives; X: [n, 3].  Returns [n, na, nb, (L+1)^2]."""
    n = len(sa)
    if nquad is None:
        nquad = L // 2 + 2
    nodes, W = _gh(nquad)
    la, lb = sa[0]["l"], sb[0]["l"]
    A = np.array([s["A"] for s in sa])
    B = np.array([s["A"] for s in sb])
    ea = np.array([s["e"] for s in sa])
    eb = np.array([s["e"] for s in sb])
    ca = np.array([s["c"] for s in sa])
    cb = np.array([s["c"] for s in sb])
    X = np.asarray(X)
    na = 1 if la == 0 else 3
    nb = 1 if lb == 0 else 3
    out = np.zeros((n, na, nb, solid.nlm(L)), dtype=np.complex128)
    AB2 = np.sum((A - B) ** 2, axis=1)
    for p in range(ea.shape[1]):
        for q in range(eb.shape[1]):
            a = ea[:, p]
            b = eb[:, q]
            pp = a + b
            P = (a[:, None] * A + b[:, None] * B) / pp[:, None]
            K = np.exp(-a * b / pp * AB2)
            pts = P[:, None, :] + nodes[None, :, :] / np.sqrt(pp)[:, None, None]
            Ov = solid.O_all(pts - X[:, None, :], L)               # [n, nq, nlm]
            fa = _cart_factor(pts, A, la)                          # [n, nq, na]
            fb = _cart_factor(pts, B, lb)                          # [n, nq, nb]
            pref = ca[:, p] * cb[:, q] * K * pp ** -1.5            # [n]
            out += pref[:, None, None, None] * np.einsum(
                "q,nqa,nqb,nql->nabl", W, fa, fb, Ov)
    return out


def contracted_norms(shells):
    """1/sqrt(self-overlap) of every contracted shell (same for x, y, z)."""
    norms = np.zeros(len(shells))
    groups = {}
    for i, s in enumerate(shells):
        groups.setdefault((s["l"], len(s["e"])), []).append(i)
    for key, ids in groups.items():
        sh = [shells[i] for i in ids]
        X = np.array([s["A"] for s in sh])
        S = pair_multipoles_raw(sh, sh, X, 0)
        norms[ids] = 1.0 / np.sqrt(S[:, 0, 0, 0].real)
    return norms


def ao_pair_multipoles(basis, pairs, centres, L, shells=None, norms=None):
    """Normalised multipole integrals for a list of shell pairs (a <= b) about
    the given per-pair centres.  Returns list of arrays [na, nb, (L+1)^2]."""
    if shells is None:
        shells = shell_data(basis)
    if norms is None:
        norms = contracted_norms(shells)
    out = [None] * len(pairs)
    groups = {}
    for k, (a, b) in enumerate(pairs):
        sa, sb = shells[a], shells[b]
        groups.setdefault((sa["l"], sb["l"], len(sa["e"]), len(sb["e"])), []).append(k)
    chunk = 4000
    for key, ks in groups.items():
        for c0 in range(0, len(ks), chunk):
            kk = ks[c0:c0 + chunk]
            sa = [shells[pairs[k][0]] for k in kk]
            sb = [shells[pairs[k][1]] for k in kk]
            X = np.array([centres[k] for k in kk])
            vals = pair_multipoles_raw(sa, sb, X, L)
            for t, k in enumerate(kk):
                a, b = pairs[k]
                out[k] = vals[t] * norms[a] * norms[b]
    return out


# ---------------------------------------------------------------------------
# Boys function
# ---------------------------------------------------------------------------

def boys(nmax: int, T):
    """F_n(T) = int_0^1 t^(2n) exp(-T t^2) dt for n = 0..nmax.

    T <= 20: series F_N(T) = exp(-T) sum_k (2T)^k / ((2N+1)(2N+3)...(2N+2k+1))
    at the top order N, then downward recursion
    F_n = (2T F_(n+1) + exp(-T)) / (2n+1).
    T > 20: F_0 = sqrt(pi/T) erf(sqrt T) / 2 and upward recursion
    F_(n+1) = ((2n+1) F_n - exp(-T)) / (2T)."""
    T = np.asarray(T, dtype=np.float64)
    out = np.zeros(T.shape + (nmax + 1,))
    eT = np.exp(-T)
    small = T <= 20.0
    if np.any(small):
        Ts = T[small]
        N = nmax
        term = np.full(Ts.shape, 1.0 / (2 * N + 1))
        acc = term.copy()
        for k in range(1, 200):
            term = term * 2.0 * Ts / (2 * N + 2 * k + 1)
            acc = acc + term
        F = np.zeros(Ts.shape + (nmax + 1,))
        F[..., N] = np.exp(-Ts) * acc
        for n in range(N - 1, -1, -1):
            F[..., n] = (2.0 * Ts * F[..., n + 1] + np.exp(-Ts)) / (2 * n + 1)
        out[small] = F
    big = ~small
    if np.any(big):
        Tb = T[big]
        F = np.zeros(Tb.shape + (nmax + 1,))
        F[..., 0] = 0.5 * np.sqrt(math.pi / Tb) * erf(np.sqrt(Tb))
        for n in range(nmax):
            F[..., n + 1] = ((2 * n + 1) * F[..., n] - eT[big]) / (2.0 * Tb)
        out[big] = F
    return out


# ---------------------------------------------------------------------------
# McMurchie-Davidson ERIs for s/p primitives
# ---------------------------------------------------------------------------

def _hermite_E(i, j, PA, PB, p):
    """1-D Hermite expansion coefficients E^{ij}_t (t = 0..i+j) of
    (x-A)^i (x-B)^j about P, without the K_AB factor; i, j <= 1.
    Arrays broadcast over PA, PB, p."""
    one = np.ones_like(PA)
    E00 = [one]
    if i == 0 and j == 0:
        return E00
    if i == 1 and j == 0:
        return [PA, 1.0 / (2 * p) * one]
    if i == 0 and j == 1:
        return [PB, 1.0 / (2 * p) * one]
    # i = j = 1: E^{11}_t from E^{10}: E^{1,1}_t = E^{10}_{t-1}/(2p) + PB E^{10}_t + (t+1) E^{10}_{t+1}
    E10 = [PA, 1.0 / (2 * p) * one]
    e0 = PB * E10[0] + 1 * E10[1]
    e1 = E10[0] / (2 * p) + PB * E10[1]
    e2 = E10[1] / (2 * p)
    return [e0, e1, e2]


def _R_table(tmax, alpha, PQ, F):
    """Hermite Coulomb integrals R^0_{tuv} for t+u+v <= tmax.
    R^n_000 = (-2 alpha)^n F_n; R^n_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X_PQ R^{n+1}_{t,u,v}."""
    R = {}
    for n in range(tmax + 1):
        R[(0, 0, 0, n)] = (-2.0 * alpha) ** n * F[..., n]

    def get(t, u, v, n):
        key = (t, u, v, n)
        if key in R:
            return R[key]
        if t > 0:
            val = PQ[..., 0] * get(t - 1, u, v, n + 1)
            if t > 1:
                val = val + (t - 1) * get(t - 2, u, v, n + 1)
        elif u > 0:
            val = PQ[..., 1] * get(t, u - 1, v, n + 1)
            if u > 1:
                val = val + (u - 1) * get(t, u - 2, v, n + 1)
        else:
            val = PQ[..., 2] * get(t, u, v - 1, n + 1)
            if v > 1:
                val = val + (v - 1) * get(t, u, v - 2, n + 1)
        R[key] = val
        return val
    return get


def _cart_powers(l, k):
    if l == 0:
        return (0, 0, 0)
    p = [0, 0, 0]
    p[k] = 1
    return tuple(p)


def eri_primitive(A, a, pa, B, b, pb, C, c, pc, D, d, pd):
    """(ab|cd) over primitive Cartesian Gaussians with powers pa..pd (each a
    3-tuple with entries 0/1), unnormalised.  Arrays broadcast."""
    p = a + b
    q = c + d
    P = (a[..., None] * A + b[..., None] * B) / p[..., None]
    Q = (c[..., None] * C + d[..., None] * D) / q[..., None]
    KAB = np.exp(-a * b / p * np.sum((A - B) ** 2, axis=-1))
    KCD = np.exp(-c * d / q * np.sum((C - D) ** 2, axis=-1))
    alpha = p * q / (p + q)
    PQ = P - Q
    ltot = sum(pa) + sum(pb) + sum(pc) + sum(pd)
    F = boys(ltot, alpha * np.sum(PQ * PQ, axis=-1))
    R = _R_table(ltot, alpha, PQ, F)
    Eab = [_hermite_E(pa[x], pb[x], P[..., x] - A[..., x], P[..., x] - B[..., x], p) for x in range(3)]
    Ecd = [_hermite_E(pc[x], pd[x], Q[..., x] - C[..., x], Q[..., x] - D[..., x], q) for x in range(3)]
    acc = 0.0
    for t, et in enumerate(Eab[0]):
        for u, eu in enumerate(Eab[1]):
            for v, ev in enumerate(Eab[2]):
                e1 = et * eu * ev
                for tau, ft in enumerate(Ecd[0]):
                    for nu, fu in enumerate(Ecd[1]):
                        for phi, fv in enumerate(Ecd[2]):
                            sgn = (-1.0) ** (tau + nu + phi)
                            acc = acc + e1 * sgn * ft * fu * fv * R(t + tau, u + nu, v + phi, 0)
    return 2.0 * math.pi ** 2.5 / (p * q * np.sqrt(p + q)) * KAB * KCD * acc


def ss_ss_closed(A, a, B, b, C, c, D, d):
    """Closed-form (ss|ss) = 2 pi^(5/2) / (p q sqrt(p+q)) K_AB K_CD F_0(rho |P-Q|^2)."""
    p = a + b
    q = c + d
    P = (a * A + b * B) / p
    Q = (c * C + d * D) / q
    KAB = math.exp(-a * b / p * float(np.sum((A - B) ** 2)))
    KCD = math.exp(-c * d / q * float(np.sum((C - D) ** 2)))
    T = p * q / (p + q) * float(np.sum((P - Q) ** 2))
    F0 = float(boys(0, np.array([T]))[0, 0])
    return 2.0 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * KAB * KCD * F0


def eri_quartets(shells, norms, quartets):
    """Contracted, normalised (ab|cd) blocks for a list of shell quartets.

    Returns a list of arrays [na, nb, nc, nd] (Cartesian components x, y, z for p)."""
    out = [None] * len(quartets)
    groups = {}
    for k, q in enumerate(quartets):
        key = tuple((shells[s]["l"], len(shells[s]["e"])) for s in q)
        groups.setdefault(key, []).append(k)
    for key, ks in groups.items():
        sh = [[shells[quartets[k][x]] for k in ks] for x in range(4)]
        cen = [np.array([s["A"] for s in shl]) for shl in sh]
        ex = [np.array([s["e"] for s in shl]) for shl in sh]
        co = [np.array([s["c"] for s in shl]) for shl in sh]
        nrm = np.prod([np.array([norms[quartets[k][x]] for k in ks]) for x in range(4)], axis=0)
        ls = [key[x][0] for x in range(4)]
        ncomp = [1 if l == 0 else 3 for l in ls]
        block = np.zeros((len(ks),) + tuple(ncomp))
        for ca in range(ncomp[0]):
            for cb in range(ncomp[1]):
                for cc in range(ncomp[2]):
                    for cd in range(ncomp[3]):
                        pw = [_cart_powers(ls[0], ca), _cart_powers(ls[1], cb),
                              _cart_powers(ls[2], cc), _cart_powers(ls[3], cd)]
                        acc = np.zeros(len(ks))
                        for i in range(ex[0].shape[1]):
                            for j in range(ex[1].shape[1]):
                                for k in range(ex[2].shape[1]):
                                    for m in range(ex[3].shape[1]):
                                        v = eri_primitive(cen[0], ex[0][:, i], pw[0], cen[1], ex[1][:, j], pw[1],
                                                          cen[2], ex[2][:, k], pw[2], cen[3], ex[3][:, m], pw[3])
                                        acc += co[0][:, i] * co[1][:, j] * co[2][:, k] * co[3][:, m] * v
                        block[:, ca, cb, cc, cd] = acc * nrm
        for t, k in enumerate(ks):
            out[k] = block[t]
    return out
