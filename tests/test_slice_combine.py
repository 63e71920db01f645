"""The conversion of exact integer group sums into a (hi, lo) pair of FP32
numbers, used by the epilogue of the sliced M2L GEMM, restated step by step
in float32 arithmetic and checked against exact rational arithmetic.

The GEMM leaves, per output, 64-bit integers vh and vl with
X = vh 2^-26 + vl 2^-(12 + 7(S-1)).  The conversion forms X 2^(12+7(S-1)) =
M 2^SH + R exactly, cuts |M|, R into non-negative chunks of at most 21 bits,
turns each into FP32 with the magic-number trick (exact), scales by exact
powers of two, adds smallest first with TwoSum and renormalises; the scaling
by 2^k comes last.  Nothing cancels, so hi + lo is within a few 2^-48 of X 2^k.
Cutting a negative sum into two's complement chunks instead (the first
version) cancels large chunks and loses about 1e-11: the second test keeps
that case as a pin of why the magnitude is cut.
"""
from fractions import Fraction

import numpy as np

f32 = np.float32


def _bits2f(i):
    return np.array([i], dtype=np.int64).astype(np.uint32).view(np.float32)[0]


def _pow2f(E):
    return f32(0.0) if E < -126 else _bits2f((min(E, 127) + 127) << 23)


def _ldexpf(x, E):
    if E >= -126:
        return f32(x * _pow2f(E))
    if E >= -252:
        return f32(f32(x * _pow2f(E + 126)) * _pow2f(-126))
    return f32(0.0)


def _two_sum(h, l, a):
    s = f32(h + a)
    bb = f32(s - h)
    return s, f32(l + f32(f32(h - f32(s - bb)) + f32(a - bb)))


def _u2f(u):
    return f32(_bits2f(0x4B000000 | int(u)) - f32(8388608.0))


def _parts(acc, S):
    vh = vl = 0
    for d in range(S):
        if d < 3:
            vh += int(acc[d]) << (7 * (2 - d))
        else:
            vl += int(acc[d]) << (7 * (S - 1 - d))
    return vh, vl


def _sum(terms):
    h, l = terms[0], f32(0)
    for a in terms[1:]:
        h, l = _two_sum(h, l, a)
    hh = f32(h + l)
    return hh, f32(l - f32(hh - h))


def combine_magnitude(acc, k, S):
    vh, vl = _parts(acc, S)
    SH = 7 * (S - 1) - 14
    M, R = vh + (vl >> SH), vl & ((1 << SH) - 1)
    neg = M < 0
    if neg:
        M = -M
        if R:
            M, R = M - 1, (1 << SH) - R
    hh, ll = _sum([_u2f(R & 0x3FFF), f32(_u2f(R >> 14) * _pow2f(14)), f32(_u2f(M & 0x1FFFFF) * _pow2f(SH)),
                   f32(_u2f((M >> 21) & 0x1FFFFF) * _pow2f(SH + 21)), f32(_u2f(M >> 42) * _pow2f(SH + 42))])
    E = k - (12 + 7 * (S - 1))
    x, y = _ldexpf(hh, E), _ldexpf(ll, E)
    return (-x, -y) if neg else (x, y)


def combine_twos_complement(acc, k, S):
    vh, vl = _parts(acc, S)

    def lo21(v, sh):
        return _u2f((v >> sh) & 0x1FFFFF)

    def top(v):
        return f32(_bits2f(0x4B400000 + (v >> 42)) - f32(12582912.0))

    el, eh = k - (12 + 7 * (S - 1)), k - 26
    return _sum([f32(lo21(vl, 0) * _pow2f(el)), f32(lo21(vl, 21) * _pow2f(el + 21)),
                 f32(top(vl) * _pow2f(el + 42)), f32(lo21(vh, 0) * _pow2f(eh)),
                 f32(lo21(vh, 21) * _pow2f(eh + 21)), f32(top(vh) * _pow2f(eh + 42))])


def _exact(acc, k, S):
    vh, vl = _parts(acc, S)
    return (Fraction(vh, 2 ** 26) + Fraction(vl, 2 ** (12 + 7 * (S - 1)))) * Fraction(2) ** k


def _rel(got, exact):
    g = Fraction(float(got[0])) + Fraction(float(got[1]))
    return 0.0 if exact == 0 and g == 0 else abs(float((g - exact) / exact))


def test_magnitude_chunks_are_accurate():
    rng = np.random.default_rng(1)
    for S in (7, 6):
        worst = 0.0
        for trial in range(3000):
            m = trial % 4
            if m == 0:
                acc = rng.integers(-2 ** 30, 2 ** 30, size=S)
            elif m == 1:
                acc = rng.integers(-2 ** 12, 2 ** 12, size=S) * rng.integers(1, 2 ** 18)
            elif m == 2:
                acc = rng.integers(-100, 100, size=S)
            else:
                acc = np.zeros(S, dtype=np.int64)
                acc[rng.integers(0, S)] = rng.integers(-2 ** 30, 2 ** 30)
                acc[rng.integers(0, S)] += rng.integers(-5, 5)
            k = int(rng.integers(-90, 30))
            ex = _exact(acc, k, S)
            got = combine_magnitude(acc, k, S)
            if ex == 0:
                assert got[0] == 0 and got[1] == 0
            else:
                worst = max(worst, _rel(got, ex))
        assert worst < 2e-14, (S, worst)


def test_twos_complement_chunks_cancel():
    acc = [-3016, 18148, -33462, 50648, 2574, -34944, -92820]
    ex = _exact(acc, -19, 7)
    assert _rel(combine_twos_complement(acc, -19, 7), ex) > 1e-12
    assert _rel(combine_magnitude(acc, -19, 7), ex) < 2e-14
