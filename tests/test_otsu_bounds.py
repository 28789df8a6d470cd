"""The pruning argument of the GPU Otsu kernel, checked on the CPU with exact
arithmetic (no GPU code involved).

The kernel evaluates Otsu's between-class variance (Segmentation section,
ref. [11]) in binary64 only at the levels whose binary32 upper bound reaches
the largest binary32 lower bound.  Its bounds, for a level with class counts
and sums (n0, s0) and (n1, s1):

    each operand converted from its 32-bit halves: RN(f(hi) * 2^32 + f(lo))
    d  = RN(RN(f(S - s0) / f(n1)) - RN(f(s0) / f(n0)))
    nn = RN(f(n0) * f(n1))
    lo = RN(RN(nn * 0.99999f) * RN(e * e)),  e = max(RN(|d| - 0.05f), 0)
    hi = RN(RN(nn * 1.00001f) * RN(g * g)),  g = RN(|d| + 0.05f)

with RN the binary32 rounding to nearest, ties to even.  This test emulates
those operations with exact rationals and one rounding per operation, and
checks on histograms of several shapes, up to 2^40 voxels, that
lo <= var <= hi for the exact rational variance at every occupied level, and
that the oracle's level (the binary64 argmax, ties to the lowest) is never
pruned: its hi is at least the largest lo.
"""
from fractions import Fraction

import numpy as np


def rn32(x):
    """Exact rational -> nearest binary32 value (ties to even), as a Fraction."""
    x = Fraction(x)
    if x == 0:
        return Fraction(0)
    sign = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    e = max(e, -126)  # subnormals share the smallest exponent
    q = Fraction(2) ** (e - 23)  # spacing of binary32 values near a
    m = a / q
    f = m.numerator // m.denominator
    r = m - f
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and f % 2 == 1):
        f += 1
    return sign * f * q


F005 = rn32(Fraction(5, 100))
F_LO = rn32(Fraction(99999, 100000))
F_HI = rn32(Fraction(100001, 100000))


def f32_u64(x):
    hi, lo = x >> 32, x & 0xFFFFFFFF
    if hi == 0:
        return rn32(lo)
    return rn32(rn32(hi) * 2 ** 32 + rn32(lo))


def bounds(n0, s0, n1, S):
    d = rn32(rn32(f32_u64(S - s0) / f32_u64(n1)) - rn32(f32_u64(s0) / f32_u64(n0)))
    nn = rn32(f32_u64(n0) * f32_u64(n1))
    e = max(rn32(abs(d) - F005), Fraction(0))
    g = rn32(abs(d) + F005)
    return rn32(rn32(nn * F_LO) * rn32(e * e)), rn32(rn32(nn * F_HI) * rn32(g * g))


def oracle_level(levels, counts):
    """Binary64 Otsu as the oracle computes it (every admissible level in
    order, strict > so ties keep the lowest)."""
    N = sum(counts)
    S = sum(u * c for u, c in zip(levels, counts))
    n0 = s0 = 0
    best, bt = None, None
    for u, c in zip(levels, counts):
        n0 += c
        s0 += u * c
        n1 = N - n0
        if n1 == 0:
            continue
        m0 = float(s0) / float(n0)
        m1 = float(S - s0) / float(n1)
        d = m1 - m0
        var = ((float(n0) * float(n1)) * d) * d
        if best is None or var > best:
            best, bt = var, u
    return bt


def check(levels, counts):
    N = sum(counts)
    S = sum(u * c for u, c in zip(levels, counts))
    n0 = s0 = 0
    LB = Fraction(0)
    his = {}
    for u, c in zip(levels, counts):
        n0 += c
        s0 += u * c
        n1 = N - n0
        if n1 == 0:
            continue
        lo, hi = bounds(n0, s0, n1, S)
        var = n0 * n1 * (Fraction(S - s0, n1) - Fraction(s0, n0)) ** 2
        assert lo <= var <= hi, (u, float(lo), float(var), float(hi))
        LB = max(LB, lo)
        his[u] = hi
    t = oracle_level(levels, counts)
    if t is not None:
        assert his[t] >= LB, (t, float(his[t]), float(LB))


def test_bounds_hold_and_never_prune_the_oracle_level():
    rng = np.random.default_rng(20261204)
    cases = []
    # two modes (background and nuclei) of a microscope frame
    for scale in (1, 1000, 3 * 10 ** 6):
        lv = np.arange(60, 900)
        c = np.round(scale * (np.exp(-((lv - 200) / 25.0) ** 2) + 0.05 * np.exp(-((lv - 700) / 60.0) ** 2))).astype(np.int64)
        cases.append((lv[c > 0], c[c > 0]))
    # flat (uniform) histograms over narrow and wide ranges
    for lo_, hi_, c in ((1000, 1100, 7), (0, 1500, 1), (30000, 30008, 5 * 10 ** 8)):
        lv = np.arange(lo_, hi_)
        cases.append((lv, np.full(len(lv), c, dtype=np.int64)))
    # random sparse levels over the whole 16-bit range, counts up to 2^31
    for _ in range(4):
        lv = np.sort(rng.choice(65536, size=300, replace=False))
        cases.append((lv, rng.integers(1, 2 ** 31, size=300)))
    # two near-equal modes far apart, 2^40 voxels in all
    lv = np.array([100, 101, 102, 60000, 60001, 60002])
    cases.append((lv, np.array([2 ** 38, 2 ** 38, 2 ** 37, 2 ** 38, 2 ** 37, 2 ** 37 + 12345])))
    # tiny cases: two, three levels, equal counts (ties)
    cases.append((np.array([0, 4, 8]), np.array([1, 2, 1])))
    cases.append((np.array([5, 65535]), np.array([3, 3])))
    for lv, c in cases:
        check([int(u) for u in lv], [int(x) for x in c])
