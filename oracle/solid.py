"""Scaled regular and irregular solid harmonics, complex, all m in [-l, l].

Definitions (Sec. I, the equations after Eq. mmexp):
    O_lm(r) = eps_m r^l / (l+|m|)!  P_{l|m|}(cos t) exp(-i m phi)
    M_lm(r) = eps_m (l-|m|)! / r^(l+1)  P_{l|m|}(cos t) exp(+i m phi)
with eps_m = 1 for m >= 0 and (-1)^m otherwise.  The paper leaves the
Condon-Shortley phase of P_lm open; this oracle uses P_lm WITHOUT it
(P_11 = +sin t).  Every identity used by the method (bipolar expansion,
M2M/M2L/L2L) holds with either choice.

Component index: lm -> l*l + l + m, so an expansion truncated at L has
(L+1)^2 complex components.

Test infrastructure only (see oracle/__init__.py).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import lpmv


def nlm(L: int) -> int:
    return (L + 1) * (L + 1)


def idx(l: int, m: int) -> int:
    return l * l + l + m


def _spherical(v):
    v = np.asarray(v, dtype=np.float64)
    x, y, z = v[..., 0], v[..., 1], v[..., 2]
    r = np.sqrt(x * x + y * y + z * z)
    with np.errstate(invalid="ignore", divide="ignore"):
        ct = np.where(r > 0, z / np.where(r > 0, r, 1.0), 1.0)
    ct = np.clip(ct, -1.0, 1.0)
    phi = np.arctan2(y, x)
    return r, ct, phi


def legendre_nocs(l: int, m: int, x):
    """Associated Legendre P_l^m(x), m >= 0, without the Condon-Shortley phase."""
    return lpmv(m, l, x) * ((-1.0) ** m)


def O_all(v, L: int) -> np.ndarray:
    """O_lm(v) for l <= L, all m; shape v.shape[:-1] + ((L+1)^2,) complex."""
    r, ct, phi = _spherical(v)
    out = np.zeros(r.shape + (nlm(L),), dtype=np.complex128)
    for l in range(L + 1):
        rl = r ** l
        for m in range(-l, l + 1):
            am = abs(m)
            eps = 1.0 if m >= 0 else (-1.0) ** am
            out[..., idx(l, m)] = (eps * rl / math.factorial(l + am)
                                   * legendre_nocs(l, am, ct) * np.exp(-1j * m * phi))
    return out


def M_all(v, L: int) -> np.ndarray:
    """M_lm(v) for l <= L, all m; v must be non-zero."""
    r, ct, phi = _spherical(v)
    out = np.zeros(r.shape + (nlm(L),), dtype=np.complex128)
    for l in range(L + 1):
        rl1 = r ** (l + 1)
        for m in range(-l, l + 1):
            am = abs(m)
            eps = 1.0 if m >= 0 else (-1.0) ** am
            out[..., idx(l, m)] = (eps * math.factorial(l - am) / rl1
                                   * legendre_nocs(l, am, ct) * np.exp(1j * m * phi))
    return out


# ---------------------------------------------------------------------------
# Translation operators as dense complex matrices (rows: output lm, cols: input l'm')
# ---------------------------------------------------------------------------

def _pairs(L):
    ls, ms = [], []
    for l in range(L + 1):
        for m in range(-l, l + 1):
            ls.append(l)
            ms.append(m)
    return np.array(ls), np.array(ms)


def m2m_matrix(d, L: int) -> np.ndarray:
    """Eq. fmm1: O_lm(Xp) = sum_{l'm'} O_{l-l',m-m'}(Xc - Xp) O_{l'm'}(Xc).

    ``d`` = Xc - Xp, shape [..., 3].  Terms with l' > l or |m-m'| > l-l'
    vanish (O_lm = 0 for |m| > l)."""
    Od = O_all(d, L)
    ls, ms = _pairs(L)
    T = np.zeros(Od.shape[:-1] + (nlm(L), nlm(L)), dtype=np.complex128)
    for a in range(nlm(L)):
        for b in range(nlm(L)):
            dl = ls[a] - ls[b]
            dm = ms[a] - ms[b]
            if dl >= 0 and abs(dm) <= dl:
                T[..., a, b] = Od[..., idx(dl, dm)]
    return T


def m2l_matrix(R, L: int, Lout: int | None = None, Lin: int | None = None) -> np.ndarray:
    """Eq. fmm2: Mcal_lm(X) = (-1)^l sum_{l'm'} M_{l+l',m+m'}(X - X') O_{l'm'}(X').

    ``R`` = X - X'.  Optional truncation of output rank (Lout) and input rank
    (Lin) below L; components above them are zero."""
    Lout = L if Lout is None else Lout
    Lin = L if Lin is None else Lin
    MR = M_all(R, 2 * L)
    ls, ms = _pairs(L)
    T = np.zeros(MR.shape[:-1] + (nlm(L), nlm(L)), dtype=np.complex128)
    for a in range(nlm(L)):
        if ls[a] > Lout:
            continue
        for b in range(nlm(L)):
            if ls[b] > Lin:
                continue
            lt = ls[a] + ls[b]
            mt = ms[a] + ms[b]
            if abs(mt) <= lt:
                T[..., a, b] = ((-1.0) ** ls[a]) * MR[..., idx(lt, mt)]
    return T


def l2l_matrix(d, L: int) -> np.ndarray:
    """Eq. fmm3: Mcal_lm(Xc) = sum_{l'm'} Mcal_{l'm'}(Xp) O_{l'-l,m'-m}(Xc - Xp).

    ``d`` = Xc - Xp.  The paper writes M for the local expansion Mcal here."""
    Od = O_all(d, L)
    ls, ms = _pairs(L)
    T = np.zeros(Od.shape[:-1] + (nlm(L), nlm(L)), dtype=np.complex128)
    for a in range(nlm(L)):
        for b in range(nlm(L)):
            dl = ls[b] - ls[a]
            dm = ms[b] - ms[a]
            if dl >= 0 and abs(dm) <= dl:
                T[..., a, b] = Od[..., idx(dl, dm)]
    return T


def bipolar(r1, X, r2, Xp, L: int) -> float:
    """Truncated Eq. mmexp: sum_{l,l' <= L} (-1)^l O_lm(r1-X) M_{l+l',m+m'}(X-X') O_l'm'(r2-X')."""
    a = O_all(np.asarray(r1) - np.asarray(X), L)
    b = O_all(np.asarray(r2) - np.asarray(Xp), L)
    T = m2l_matrix(np.asarray(X) - np.asarray(Xp), L)
    return complex(a @ (T @ b))
