"""The error-free splitting used by every integer-slice GEMM of the
FP64-accurate form (steps (a), (e) and M2L), restated with Python integers
and checked against exact rationals.

An entry x with |x| < 1 (after its row's power-of-two scaling) is rounded to
r = round(x 2^55), computed from the FP64 bits with integer operations, and
cut into S slices: q_s = round(r_s 2^-(49 - 7 s)), r_{s+1} = r_s - q_s 2^(49 - 7 s).
Claims pinned here: every slice is an integer with |q_s| <= 64 (exact in
FP16, products below 2^12 in magnitude); x = sum_s q_s 2^-(6 + 7 s) + e with
|e| <= 2^-7S + 2^-56 (2^-49 + 2^-56 for S = 7); and the chunk of 512 K values
keeps every group sum of at most 7 slice pairs below 2^24, exact in the
tensor core's FP32 accumulator.
"""
import struct
from fractions import Fraction

import numpy as np


def _fixed(v, t):
    """round(v 2^t) from the bits of v, halves away from zero."""
    bits = struct.unpack("<q", struct.pack("<d", v))[0]
    ef = (bits >> 52) & 0x7FF
    mant = bits & ((1 << 52) - 1)
    E = -1074
    if ef != 0:
        mant |= 1 << 52
        E = ef - 1075
    sh = E + t
    if sh >= 0:
        r = mant << min(sh, 10)
    elif sh > -60:
        r = (mant + (1 << (-sh - 1))) >> (-sh)
    else:
        r = 0
    return -r if bits < 0 else r


def _slices(x, S):
    r = _fixed(x, 55)
    q = []
    for s in range(S):
        sh = 49 - 7 * s
        qs = (r + (1 << (sh - 1))) >> sh
        r -= qs << sh
        q.append(qs)
    return q, r


def test_fixed_point_rounding():
    rng = np.random.default_rng(3)
    for x in list(rng.uniform(-1, 1, 2000)) + [0.0, -0.0, 1 - 2 ** -53, -(1 - 2 ** -53), 2 ** -60, 5e-324]:
        r = _fixed(float(x), 55)
        exact = Fraction(float(x)) * 2 ** 55
        assert abs(Fraction(r) - exact) <= Fraction(1, 2)


def test_slices_are_small_and_reconstruct():
    rng = np.random.default_rng(4)
    xs = list(rng.uniform(-1, 1, 3000)) + list(rng.uniform(-1, 1, 500) * 2.0 ** -rng.integers(1, 60, 500))
    xs += [1 - 2 ** -53, -(1 - 2 ** -53), 0.5, -0.5, 2 ** -49, 63.5 / 64]
    for S in (7, 6, 4):
        bound = Fraction(1, 2 ** (7 * S)) + Fraction(1, 2 ** 56)
        for x in xs:
            q, r = _slices(float(x), S)
            assert all(abs(v) <= 64 for v in q)
            approx = sum(Fraction(v, 2 ** (6 + 7 * s)) for s, v in enumerate(q))
            assert approx + Fraction(r, 2 ** 55) == Fraction(_fixed(float(x), 55), 2 ** 55)
            assert abs(Fraction(float(x)) - approx) <= bound


def test_group_sums_fit_fp32():
    # a group d = s + t holds at most 7 slice pairs (S = 7), each product below
    # 2^12 in magnitude; a chunk is 16 stages of 32 K values
    assert 7 * 64 * 64 * (16 * 32) < 2 ** 24
    # int32 sums of the chunk sums over at most 127 chunks
    assert 127 * (2 ** 24 - 1) < 2 ** 31
