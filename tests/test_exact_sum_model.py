"""CPU model of the exact integer dot products that the matrix-powers level
and the recovery run on GB300's integer pipes (paper eq. rho and eq. coords
evaluated without binary64 FMAs), checked against exact rational arithmetic.

The arithmetic, restated here in Python integers: a binary64 v splits into
signed limbs a (31 bits of the significand) and b (22 bits) with v's sign and
an exponent e, v = (a 2^22 + b) 2^(e - 1075); a product of two split values
is ac + floor((ad + bc) / 2^22), the product over 2^44 with an error below 2.
Two ways to add such products are used:
  aligned sum   every product shifted (toward -infinity) to the largest
                exponent sum Em of the dot product with 3 guard bits; the
                sum is within 1.25 K 2^-57 of the largest |term| for K <= 8
                terms, then rounded once to nearest binary64;
  online sum    (OnlineSum<H>) each product rounded to nearest at the
                largest exponent sum seen so far, the running sum rounded to
                nearest when that grows; within m (1 + 2^(1-H)) 2^(H-60) of
                the largest |term| for m <= 2^H terms, then rounded once.
Each bound is checked on seeded inputs spread over many binades, on
cancelling sums and on exact zeros; the 64-bit sums never overflow.
"""
import struct
from fractions import Fraction

import numpy as np
import pytest

U = Fraction(1, 2 ** 53)


def to_limbs(v: float, neg: bool = False):
    bits = struct.unpack("<Q", struct.pack("<d", v))[0]
    hi, lo = (bits >> 32) ^ (0x80000000 if neg else 0), bits & 0xFFFFFFFF
    e = (hi >> 20) & 0x7FF
    assert e != 0x7FF
    m = (((hi & 0xFFFFF) | (0x100000 if e else 0)) << 32) | lo
    s = -1 if hi >> 31 else 1
    return s * (m >> 22), s * (m & 0x3FFFFF), max(e, 1)


def value(l):
    a, b, e = l
    return Fraction(a * 2 ** 22 + b) * Fraction(2) ** (e - 1075)


def limb_product(c, y):
    return c[0] * y[0] + ((c[0] * y[1] + c[1] * y[0]) >> 22)


def shift_round(x, d):
    return ((x >> (d - 1)) + 1) >> 1


def to_binary64(S, Em):
    """S 2^(Em - 2103) rounded to nearest (ties to even); None outside the normal range."""
    if S == 0:
        return 0.0
    be = abs(S).bit_length() - 1 + Em - 1080
    if be <= 0 or be >= 2047:
        return None
    return float(Fraction(S) * Fraction(2) ** (Em - 2103))


def aligned_sum(cs, ys):
    Em = max(c[2] + y[2] for c, y in zip(cs, ys))
    S = sum(limb_product(c, y) >> (Em - (c[2] + y[2]) + 3) for c, y in zip(cs, ys))
    assert -2 ** 63 <= S < 2 ** 63
    return S, Fraction(S) * Fraction(2) ** (Em - 2103), to_binary64(S, Em)


def online_sum(cs, ys, H):
    S, E = 0, 0
    for c, y in zip(cs, ys):
        Ej = c[2] + y[2]
        if Ej > E:
            S = shift_round(S, Ej - E)
            E = Ej
        S += shift_round(limb_product(c, y), E - Ej + H)
        assert -2 ** 63 <= S < 2 ** 63
    return S, Fraction(S) * Fraction(2) ** (E - 2106 + H), to_binary64(S, E + H - 3)


def spread(rng, k, lo=-60, hi=60):
    v = rng.standard_normal(k) * 2.0 ** rng.integers(lo, hi, k)
    v[rng.random(k) < 0.1] = 0.0
    return v


def test_limb_split_is_exact():
    rng = np.random.default_rng(1)
    vals = list(spread(rng, 500, -1000, 1000)) + [0.0, -0.0, 5e-324, -2.2250738585072014e-308, 1.7976931348623157e308]
    for v in vals:
        for neg in (False, True):
            a, b, e = to_limbs(float(v), neg)
            assert abs(a) < 2 ** 31 and abs(b) < 2 ** 22
            assert value((a, b, e)) == (-1 if neg else 1) * Fraction(float(v))


def test_limb_product_error_below_two_units():
    rng = np.random.default_rng(2)
    x, y = spread(rng, 2000, -300, 300), spread(rng, 2000, -300, 300)
    for u, v in zip(x, y):
        c, d = to_limbs(float(u)), to_limbs(float(v))
        exact = Fraction((c[0] * 2 ** 22 + c[1]) * (d[0] * 2 ** 22 + d[1]), 2 ** 44)
        P = limb_product(c, d)
        assert abs(P - exact) < 2 and abs(P) < 2 ** 62 + 2 ** 33


def _terms(rng, K, mode):
    if mode == "spread":
        return spread(rng, K), spread(rng, K)
    if mode == "cancel":     # a stencil row applied to a constant: sum = rounding residue of the diagonal
        k = np.exp(rng.standard_normal(K - 1))
        d = 0.0
        for t in k:
            d += t
        c = np.concatenate([[d], -k])
        return c, np.full(K, 1.3)
    if mode == "wide":       # one term far above the rest
        c, y = spread(rng, K), spread(rng, K)
        c[0], y[0] = 2.0 ** 200, 3.0
        return c, y
    raise ValueError(mode)


@pytest.mark.parametrize("mode", ["spread", "cancel", "wide"])
@pytest.mark.parametrize("K", [5, 7, 8])
def test_aligned_sum_bound(K, mode):
    rng = np.random.default_rng(10 * K + len(mode))
    for _ in range(300):
        c, y = _terms(rng, K, mode)
        cs, ys = [to_limbs(float(t)) for t in c], [to_limbs(float(t)) for t in y]
        prods = [Fraction(float(a)) * Fraction(float(b)) for a, b in zip(c, y)]
        exact, big = sum(prods, Fraction(0)), max(abs(p) for p in prods)
        S, before, got = aligned_sum(cs, ys)
        if big == 0:
            assert S == 0 and got == 0.0
            continue
        assert abs(before - exact) <= Fraction(5, 4) * K * Fraction(1, 2 ** 57) * big
        if got is not None:
            assert abs(Fraction(got) - exact) <= U * abs(exact) + Fraction(6, 10) * U * big


@pytest.mark.parametrize("mode", ["spread", "cancel", "wide"])
@pytest.mark.parametrize("H,m", [(3, 8), (3, 5), (6, 34)])
def test_online_sum_bound(H, m, mode):
    rng = np.random.default_rng(100 * H + m + len(mode))
    for _ in range(200):
        c, y = _terms(rng, m, mode)
        order = rng.permutation(m)   # the bound holds whatever order the exponents arrive in
        c, y = c[order], y[order]
        cs, ys = [to_limbs(float(t)) for t in c], [to_limbs(float(t)) for t in y]
        prods = [Fraction(float(a)) * Fraction(float(b)) for a, b in zip(c, y)]
        exact, big = sum(prods, Fraction(0)), max(abs(p) for p in prods)
        S, before, got = online_sum(cs, ys, H)
        if big == 0:
            assert S == 0 and got == 0.0
            continue
        bound = m * (1 + Fraction(1, 2 ** (H - 1))) * Fraction(2) ** (H - 60) * big
        assert abs(before - exact) <= bound
        if got is not None:
            assert abs(Fraction(got) - exact) <= U * abs(exact) + bound * (1 + U)


def test_rounding_is_to_nearest_even():
    # S 2^(Em - 2103) with Em = 2103: the integer S itself
    for S in (2 ** 53 + 1, 2 ** 53 + 3, -(2 ** 54 + 2), 2 ** 62 + 2 ** 9, 2 ** 62 + 3 * 2 ** 9, 7):
        assert to_binary64(S, 2103) == float(S)   # Python's int -> float rounds to nearest even
    assert to_binary64(2 ** 53 + 1, 2103) == float(2 ** 53)
    assert to_binary64(2 ** 53 + 3, 2103) == float(2 ** 53 + 4)
    assert to_binary64(1, 1080) is None            # below the normal range


def test_shift_round_is_to_nearest():
    """The online sum's re-alignment rounds to nearest (ties toward +infinity):
    its bound counts half a unit per rounding, not a whole one."""
    rng = np.random.default_rng(5)
    for x in [int(t) for t in rng.integers(-2 ** 62, 2 ** 62, 2000)] + [5, -5, 6, -6, 7, -7]:
        for d in (1, 2, 3, 17, 40):
            q = Fraction(x, 2 ** d)
            r = shift_round(x, d)
            assert abs(r - q) <= Fraction(1, 2) and (abs(r - q) < Fraction(1, 2) or r > q)
