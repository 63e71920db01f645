"""Pins for the oracle's Gaussian integrals.

* Boys function against mpmath's confluent hypergeometric form.
* AO-pair multipoles (Sec. II, multipole-integral definition): for an s-s
  product the integrand is a Gaussian times a harmonic polynomial, and by the
  mean-value property of harmonic functions its integral is
  (pi/p)^(3/2) O_lm(P - X) exactly.  p functions are (1/2a) d/dA of s
  functions, checked by central differences.  The monopole equals the overlap
  computed independently by the input generator.
* ERIs (Eq. erib): (ss|ss) closed form; p functions by finite differences of
  s integrals with respect to the centre; the far-separated limit
  (ss|ss) -> S_ab S_cd / R.
"""
import math

import numpy as np
import pytest

from oracle import gauss, solid
from paper_1708_05353_gb300 import inputs

rng = np.random.default_rng(2024)


def test_boys_vs_mpmath():
    mpmath = pytest.importorskip("mpmath")
    Ts = np.array([0.0, 1e-8, 1e-3, 0.3, 1.0, 3.7, 9.9, 15.0, 19.99, 20.01, 27.0, 60.0, 300.0])
    F = gauss.boys(6, Ts)
    for t, T in enumerate(Ts):
        for n in range(7):
            ref = float(mpmath.hyp1f1(n + 0.5, n + 1.5, -T) / (2 * n + 1))
            assert F[t, n] == pytest.approx(ref, rel=2e-14, abs=1e-300)


def _shell(A, l, e, c):
    e = np.atleast_1d(np.asarray(e, float))
    c = np.atleast_1d(np.asarray(c, float))
    n = (2 * e / math.pi) ** 0.75
    if l == 1:
        n = n * 2 * np.sqrt(e)
    return dict(A=np.asarray(A, float), l=l, e=e, c=c * n, ao=0, nao=1 if l == 0 else 3)


def _ss_mean_value(A, a, B, b, X, L):
    """(pi/p)^(3/2) K O_lm(P - X) for unnormalised primitives."""
    p = a + b
    P = (a * A + b * B) / p
    K = math.exp(-a * b / p * float(np.sum((A - B) ** 2)))
    return (math.pi / p) ** 1.5 * K * solid.O_all(P - X, L)


@pytest.mark.parametrize("L", [0, 2, 5, 10])
def test_ss_multipoles_mean_value(L):
    for _ in range(3):
        A, B, X = rng.normal(size=(3, 3)) * 1.5
        a, b = rng.uniform(0.2, 4.0, size=2)
        sa = _shell(A, 0, [a], [1.0])
        sb = _shell(B, 0, [b], [1.0])
        got = gauss.pair_multipoles_raw([sa], [sb], X[None], L)[0, 0, 0]
        ref = _ss_mean_value(A, a, B, b, X, L) * sa["c"][0] * sb["c"][0]
        np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


def test_p_multipoles_by_centre_derivative():
    """(x-A_x) exp(-a|r-A|^2) = (1/2a) d/dA_x exp(-a|r-A|^2)."""
    L = 4
    h = 1e-5
    A, B, X = rng.normal(size=(3, 3))
    a, b = 1.3, 0.7
    sp = _shell(A, 1, [a], [1.0])
    ss = _shell(B, 0, [b], [1.0])
    pp_ = _shell(B, 1, [b], [1.0])
    got_ps = gauss.pair_multipoles_raw([sp], [ss], X[None], L)[0]          # [3, 1, nlm]
    got_pp = gauss.pair_multipoles_raw([sp], [pp_], X[None], L)[0]         # [3, 3, nlm]
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        d = (_ss_mean_value(A + e, a, B, b, X, L) - _ss_mean_value(A - e, a, B, b, X, L)) / (2 * h)
        ref = d / (2 * a) * sp["c"][0] * ss["c"][0]
        np.testing.assert_allclose(got_ps[k, 0], ref, rtol=1e-6, atol=1e-8)
        for q in range(3):
            f = np.zeros(3)
            f[q] = h
            dd = (_ss_mean_value(A + e, a, B + f, b, X, L) - _ss_mean_value(A + e, a, B - f, b, X, L)
                  - _ss_mean_value(A - e, a, B + f, b, X, L) + _ss_mean_value(A - e, a, B - f, b, X, L)) / (4 * h * h)
            ref2 = dd / (4 * a * b) * sp["c"][0] * pp_["c"][0]
            np.testing.assert_allclose(got_pp[k, q], ref2, rtol=2e-4, atol=1e-5)


def test_quadrature_is_exact():
    """More nodes give the same integrals: the quadrature is exact, not converged."""
    L = 6
    A, B, X = rng.normal(size=(3, 3))
    sa = _shell(A, 1, [2.0, 0.4], [0.6, 0.5])
    sb = _shell(B, 1, [1.1], [1.0])
    r1 = gauss.pair_multipoles_raw([sa], [sb], X[None], L)
    r2 = gauss.pair_multipoles_raw([sa], [sb], X[None], L, nquad=L // 2 + 5)
    np.testing.assert_allclose(r1, r2, rtol=1e-12, atol=1e-14)


def test_monopole_is_input_overlap():
    s = inputs.small_sp(natom=4)
    S = inputs.overlap_matrix(s.basis)
    shells = gauss.shell_data(s.basis)
    norms = gauss.contracted_norms(shells)
    aoff = s.basis.shell_ao_offset
    pairs = [(a, b) for a in range(s.basis.nshell) for b in range(a, s.basis.nshell)]
    X = rng.normal(size=(len(pairs), 3))
    Om = gauss.ao_pair_multipoles(s.basis, pairs, X, 1, shells, norms)
    for (a, b), O in zip(pairs, Om):
        blk = S[aoff[a]:aoff[a + 1], aoff[b]:aoff[b + 1]]
        np.testing.assert_allclose(O[:, :, 0].real, blk, rtol=1e-12, atol=1e-14)


def _eri_prims(A, a, pa, B, b, pb, C, c, pc, D, d, pd):
    f = lambda x: np.asarray([x], float)
    return float(gauss.eri_primitive(A[None], f(a), pa, B[None], f(b), pb,
                                     C[None], f(c), pc, D[None], f(d), pd)[0])


def test_ssss_closed_form():
    s0 = (0, 0, 0)
    for _ in range(5):
        A, B, C, D = rng.normal(size=(4, 3)) * 2
        a, b, c, d = rng.uniform(0.1, 5, size=4)
        got = _eri_prims(A, a, s0, B, b, s0, C, c, s0, D, d, s0)
        assert got == pytest.approx(gauss.ss_ss_closed(A, a, B, b, C, c, D, d), rel=1e-13)
    # all on one centre, F_0(0) = 1
    A = np.zeros(3)
    got = _eri_prims(A, 1.0, s0, A, 1.0, s0, A, 1.0, s0, A, 1.0, s0)
    assert got == pytest.approx(2 * math.pi ** 2.5 / (2 * 2 * math.sqrt(4)), rel=1e-14)


def test_ssss_far_limit():
    s0 = (0, 0, 0)
    A = np.zeros(3)
    B = np.array([0.3, 0, 0])
    C = np.array([200.0, 10.0, 0.0])
    D = C + np.array([0, 0.4, 0])
    a, b, c, d = 1.0, 0.7, 1.3, 0.5
    Sab = (math.pi / (a + b)) ** 1.5 * math.exp(-a * b / (a + b) * 0.09)
    Scd = (math.pi / (c + d)) ** 1.5 * math.exp(-c * d / (c + d) * 0.16)
    P = (a * A + b * B) / (a + b)
    Q = (c * C + d * D) / (c + d)
    got = _eri_prims(A, a, s0, B, b, s0, C, c, s0, D, d, s0)
    assert got == pytest.approx(Sab * Scd / np.linalg.norm(P - Q), rel=1e-12)


@pytest.mark.parametrize("slot", [0, 1, 2, 3])
def test_p_eri_by_centre_derivative(slot):
    """(p_k ...| ...) = (1/2 alpha) d/dCentre_k of the s integral, any slot."""
    s0 = (0, 0, 0)
    cen = list(rng.normal(size=(4, 3)) * 1.5)
    ex = list(rng.uniform(0.3, 3.0, size=4))
    h = 1e-5
    for k in range(3):
        pw = [s0] * 4
        pk = [0, 0, 0]
        pk[k] = 1
        pw[slot] = tuple(pk)
        got = _eri_prims(cen[0], ex[0], pw[0], cen[1], ex[1], pw[1], cen[2], ex[2], pw[2], cen[3], ex[3], pw[3])
        cp = [c.copy() for c in cen]
        cm = [c.copy() for c in cen]
        cp[slot][k] += h
        cm[slot][k] -= h
        fp = _eri_prims(cp[0], ex[0], s0, cp[1], ex[1], s0, cp[2], ex[2], s0, cp[3], ex[3], s0)
        fm = _eri_prims(cm[0], ex[0], s0, cm[1], ex[1], s0, cm[2], ex[2], s0, cm[3], ex[3], s0)
        ref = (fp - fm) / (2 * h) / (2 * ex[slot])
        assert got == pytest.approx(ref, rel=1e-6, abs=1e-9)


def test_pp_pp_eri_by_mixed_derivative():
    """(p_x p_y | p_z p_x) from four centre derivatives of (ss|ss)."""
    s0 = (0, 0, 0)
    cen = list(rng.normal(size=(4, 3)) * 1.2)
    ex = [1.1, 0.8, 1.4, 0.6]
    comps = [0, 1, 2, 0]
    pw = []
    for k in comps:
        p = [0, 0, 0]
        p[k] = 1
        pw.append(tuple(p))
    got = _eri_prims(cen[0], ex[0], pw[0], cen[1], ex[1], pw[1], cen[2], ex[2], pw[2], cen[3], ex[3], pw[3])
    h = 2e-3
    acc = 0.0
    for signs in np.ndindex(2, 2, 2, 2):
        cc = [c.copy() for c in cen]
        sg = 1.0
        for slot, s in enumerate(signs):
            d = h if s == 0 else -h
            cc[slot][comps[slot]] += d
            sg *= 1.0 if s == 0 else -1.0
        acc += sg * _eri_prims(cc[0], ex[0], s0, cc[1], ex[1], s0, cc[2], ex[2], s0, cc[3], ex[3], s0)
    ref = acc / (2 * h) ** 4 / (16 * ex[0] * ex[1] * ex[2] * ex[3])
    assert got == pytest.approx(ref, rel=1e-4)
