"""Pins for the oracle's solid harmonics and translation operators.

Each check is fixed by mathematics independent of the oracle's own code path
(scipy lpmv): hand-derived low-order closed forms, the Legendre addition
theorem, harmonicity and homogeneity, and the exactness / convergence of the
translation identities (Sec. I, Eq. mmexp; Sec. II, Eqs. fmm1-fmm3)."""
import math

import numpy as np
import pytest
from scipy.special import eval_legendre

from oracle import solid

rng = np.random.default_rng(12345)


def test_low_order_closed_forms():
    for _ in range(20):
        v = rng.normal(size=3)
        x, y, z = v
        r = np.linalg.norm(v)
        O = solid.O_all(v, 2)
        M = solid.M_all(v, 1)
        assert O[solid.idx(0, 0)] == pytest.approx(1.0)
        assert O[solid.idx(1, 0)] == pytest.approx(z)
        assert O[solid.idx(1, 1)] == pytest.approx((x - 1j * y) / 2)
        assert O[solid.idx(1, -1)] == pytest.approx(-(x + 1j * y) / 2)
        assert O[solid.idx(2, 0)] == pytest.approx((2 * z * z - x * x - y * y) / 4)
        assert O[solid.idx(2, 1)] == pytest.approx(z * (x - 1j * y) / 2)
        assert O[solid.idx(2, 2)] == pytest.approx((x - 1j * y) ** 2 / 8)
        assert M[solid.idx(0, 0)] == pytest.approx(1 / r)
        assert M[solid.idx(1, 0)] == pytest.approx(z / r ** 3)
        assert M[solid.idx(1, 1)] == pytest.approx((x + 1j * y) / r ** 3)


def test_conjugate_symmetry_and_homogeneity():
    L = 8
    v = rng.normal(size=3)
    O = solid.O_all(v, L)
    M = solid.M_all(v, L)
    O2 = solid.O_all(2.5 * v, L)
    M2 = solid.M_all(2.5 * v, L)
    for l in range(L + 1):
        for m in range(1, l + 1):
            assert O[solid.idx(l, -m)] == pytest.approx((-1) ** m * np.conj(O[solid.idx(l, m)]))
            assert M[solid.idx(l, -m)] == pytest.approx((-1) ** m * np.conj(M[solid.idx(l, m)]))
        for m in range(-l, l + 1):
            assert O2[solid.idx(l, m)] == pytest.approx(2.5 ** l * O[solid.idx(l, m)], rel=1e-12)
            assert M2[solid.idx(l, m)] == pytest.approx(2.5 ** (-l - 1) * M[solid.idx(l, m)], rel=1e-12)


def test_harmonic():
    """Regular and irregular solid harmonics solve Laplace's equation."""
    L = 6
    v = rng.normal(size=3) + np.array([0, 0, 1.5])
    h = 1e-3
    lapO = -6 * solid.O_all(v, L)
    lapM = -6 * solid.M_all(v, L)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        lapO = lapO + solid.O_all(v + e, L) + solid.O_all(v - e, L)
        lapM = lapM + solid.M_all(v + e, L) + solid.M_all(v - e, L)
    scaleO = np.abs(solid.O_all(v, L)).max()
    scaleM = np.abs(solid.M_all(v, L)).max()
    assert np.abs(lapO).max() / h ** 2 < 1e-4 * scaleO
    assert np.abs(lapM).max() / h ** 2 < 1e-4 * scaleM


@pytest.mark.parametrize("l", range(0, 9))
def test_legendre_addition_theorem(l):
    """sum_m O_lm(r) M_lm(R) = r^l / R^(l+1) P_l(cos gamma)."""
    for _ in range(5):
        r = rng.normal(size=3)
        R = rng.normal(size=3) * 3
        O = solid.O_all(r, l)
        M = solid.M_all(R, l)
        s = sum(O[solid.idx(l, m)] * M[solid.idx(l, m)] for m in range(-l, l + 1))
        nr, nR = np.linalg.norm(r), np.linalg.norm(R)
        ref = nr ** l / nR ** (l + 1) * eval_legendre(l, r @ R / (nr * nR))
        assert abs(s.imag) < 1e-12 * max(1, abs(ref))
        assert s.real == pytest.approx(ref, rel=1e-10, abs=1e-14)


def test_bipolar_expansion_converges():
    """Eq. mmexp: geometric convergence to 1/|r1-r2| for separated points,
    error below C rho^(L+1), rho = (|a|+|b|)/|X-X'|."""
    for trial in range(4):
        X = np.zeros(3)
        Xp = rng.normal(size=3)
        Xp = 6.0 * Xp / np.linalg.norm(Xp)
        a = rng.normal(size=3)
        a = 0.6 * a / np.linalg.norm(a)
        b = rng.normal(size=3)
        b = 0.6 * b / np.linalg.norm(b)
        exact = 1.0 / np.linalg.norm((X + a) - (Xp + b))
        rho = 1.2 / 6.0
        errs = []
        for L in (1, 2, 4, 6, 8, 10):
            v = solid.bipolar(X + a, X, Xp + b, Xp, L)
            assert abs(v.imag) < 1e-14
            err = abs(v.real - exact)
            errs.append(err)
            assert err <= 4.0 * rho ** (L + 1) / (1 - rho) / 6.0 + 1e-15
        assert errs[-1] < 1e-9


def test_m2m_exact():
    """Eq. fmm1 is an exact finite identity: O(r - Xp) = T(Xc - Xp) O(r - Xc)."""
    L = 7
    for _ in range(5):
        Xc, Xp, r = rng.normal(size=(3, 3))
        T = solid.m2m_matrix(Xc - Xp, L)
        np.testing.assert_allclose(T @ solid.O_all(r - Xc, L), solid.O_all(r - Xp, L),
                                   rtol=1e-12, atol=1e-13)


def test_l2l_exact():
    """Eq. fmm3 re-centres a truncated local expansion exactly:
    sum_lm O_lm(r - Xp) Mcal_lm(Xp) = sum_lm O_lm(r - Xc) Mcal_lm(Xc)."""
    L = 7
    for _ in range(5):
        Xc, Xp, r = rng.normal(size=(3, 3))
        loc = rng.normal(size=solid.nlm(L)) + 1j * rng.normal(size=solid.nlm(L))
        T = solid.l2l_matrix(Xc - Xp, L)
        lhs = solid.O_all(r - Xp, L) @ loc
        rhs = solid.O_all(r - Xc, L) @ (T @ loc)
        assert rhs == pytest.approx(lhs, rel=1e-11, abs=1e-12)


def test_m2l_potential_of_point_charge():
    """Eq. fmm2 applied to the multipoles of a point charge q at X'+b gives a
    local expansion whose potential at X+a converges to q/|X+a-X'-b|."""
    q = 0.7
    X = np.zeros(3)
    Xp = np.array([4.0, -3.0, 2.0])
    a = np.array([0.3, 0.2, -0.4])
    b = np.array([-0.2, 0.5, 0.1])
    exact = q / np.linalg.norm(X + a - Xp - b)
    prev = None
    for L in (2, 4, 6, 8, 10):
        Omul = q * solid.O_all(b, L)
        loc = solid.m2l_matrix(X - Xp, L) @ Omul
        pot = solid.O_all(a, L) @ loc
        err = abs(pot - exact)
        if prev is not None:
            assert err < prev
        prev = err
    assert prev < 1e-8


def test_m2l_truncation_restricts_ranks():
    L = 5
    R = np.array([3.0, 1.0, -2.0])
    T = solid.m2l_matrix(R, L, Lout=2, Lin=3)
    ls = np.array([l for l in range(L + 1) for m in range(-l, l + 1)])
    assert np.all(T[ls > 2, :] == 0)
    assert np.all(T[:, ls > 3] == 0)
    full = solid.m2l_matrix(R, L)
    sel = (ls[:, None] <= 2) & (ls[None, :] <= 3)
    np.testing.assert_array_equal(T[sel], full[sel])
