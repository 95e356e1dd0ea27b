"""Exact-arithmetic model of the tensor-core Grams' digit schemes (no GPU).

The library writes each binary64 value y of a basis column as the 60-bit
integer F = round(|y| 2^(1082 - ce)) (ce: the biased exponent of the
column's largest value in its chunk) and splits F into P digits of b bits,
F = sum_t d_t 2^(b (P - 1 - t)): gram_mode 2 takes P = 12 five-bit digits,
gram_mode 3 P = 10 six-bit digits.  It forms the digit products of the plane
pairs s + t <= P - 1 exactly and adds them with the weights
2^(ce_i + ce_j - 2164 + b (2P - 2 - s - t)).  These tests restate that
arithmetic with Python integers and fractions (nothing from the CUDA path)
and check, for both schemes, the claims the kernels' accuracy rests on:
digits exact within 2^7 of the column's largest value, the rounding of F at
2^-60 of it, the dropped pairs below 2^-53 of the product of the two column
maxima per row, the binary32 block sums below 2^24, G within
2^-53 ||y_i|| ||y_j|| of the exact Gram (normwise; binary64 FMAs are bounded
by n 2^-53 ||y_i|| ||y_j||), and the componentwise caveat.
"""
from __future__ import annotations

import math
import struct
from fractions import Fraction

import numpy as np
import pytest

# (planes, bits per digit, rows per exact binary32 block sum, digit pairs per sum)
SCHEMES = {"gram_mode 2": (12, 5, 1024, 12), "gram_mode 3": (10, 6, 4096, 1)}
scheme = pytest.mark.parametrize("name", sorted(SCHEMES))


def biased_exponent(y: float) -> int:
    e = (struct.unpack("<Q", struct.pack("<d", y))[0] >> 52) & 0x7FF
    return max(e, 1)


def fixed(y: float, ce: int) -> int:
    """round(|y| 2^(1082 - ce)) from the exact binary value of y."""
    v = Fraction(abs(y)) * Fraction(2) ** (1082 - ce)
    return math.floor(v + Fraction(1, 2))


def digits(F: int, planes: int, bits: int) -> list[int]:
    return [(F >> (bits * (planes - 1 - t))) & ((1 << bits) - 1) for t in range(planes)]


def digit_gram(Y: np.ndarray, planes: int, bits: int) -> list[list[Fraction]]:
    """G by the truncated digit products, exactly (one scale chunk)."""
    n, c = Y.shape
    ce = [max(biased_exponent(float(v)) for v in Y[:, j]) for j in range(c)]
    D = [[(math.copysign(1, Y[r, j]), digits(fixed(float(Y[r, j]), ce[j]), planes, bits)) for j in range(c)]
         for r in range(n)]
    G = [[Fraction(0)] * c for _ in range(c)]
    for i in range(c):
        for j in range(i, c):
            acc = 0
            for r in range(n):
                si, di = D[r][i]
                sj, dj = D[r][j]
                row = 0
                for s in range(planes):
                    for t in range(planes - s):
                        row += di[s] * dj[t] * 2 ** (bits * (2 * planes - 2 - s - t))
                acc += int(si * sj) * row
            G[i][j] = G[j][i] = Fraction(acc) * Fraction(2) ** (ce[i] + ce[j] - 2164)
    return G


@scheme
def test_digits_reconstruct_and_round(name):
    planes, bits, _, _ = SCHEMES[name]
    rng = np.random.default_rng(5)
    col = rng.standard_normal(200) * np.exp2(rng.integers(-20, 3, 200))
    ce = max(biased_exponent(float(v)) for v in col)
    unit = Fraction(2) ** (ce - 1082)           # value of one unit of F
    top = Fraction(2) ** (ce - 1023 + 1)        # 2^(e_max + 1) > every |y|
    for y in col:
        F = fixed(float(y), ce)
        assert 0 <= F < 2 ** 60
        assert F == sum(d * 2 ** (bits * (planes - 1 - t)) for t, d in enumerate(digits(F, planes, bits)))
        err = abs(Fraction(abs(float(y))) - F * unit)
        if biased_exponent(float(y)) >= ce - 7:
            assert err == 0                     # within 2^7 of the largest: all 53 bits kept
        assert err <= unit / 2                  # else rounded at bit 60 of the scale
        assert unit / 2 <= top * Fraction(2) ** -60


@scheme
def test_dropped_pairs_below_binary64_rounding(name):
    """The digit pairs s + t >= P weigh less than 2^-53 of the product of the
    two column maxima (per row)."""
    planes, bits, _, _ = SCHEMES[name]
    dmax = (1 << bits) - 1
    dropped = sum(dmax * dmax * 2 ** (bits * (2 * planes - 2 - u)) * (2 * planes - 1 - u)
                  for u in range(planes, 2 * planes - 1))
    largest = 2 ** 59 * 2 ** 59                 # F of a column maximum is at least 2^59
    assert Fraction(dropped, largest) < Fraction(1, 2 ** 53)


@scheme
def test_block_sums_stay_exact_in_binary32(name):
    """gram_mode 2 sums all pairs of one u (up to 12) over 1024 rows, gram_mode 3
    one pair over a 4096-row chunk: with digits below 2^b every partial sum is
    an integer below 2^24 (exact in binary32), and twice the rows would not
    be."""
    planes, bits, rows, pairs = SCHEMES[name]
    dmax = (1 << bits) - 1
    assert rows * pairs * dmax * dmax < 2 ** 24
    assert 2 * rows * pairs * dmax * dmax >= 2 ** 24


@scheme
@pytest.mark.parametrize("seed,spread", [(1, 0), (2, 8), (3, 40), (4, 60)])
def test_digit_gram_normwise_within_binary64(name, seed, spread):
    """On small column sets (rows of mixed sizes up to 2^+-60 apart, columns
    of different scales) the digit Gram's error is below 2^-53 ||y_i|| ||y_j||
    (binary64 FMAs are only bounded by n 2^-53 ||y_i|| ||y_j||) and below
    n 2^-56 max_i max_j (the dropped pairs, about 2^-56.5 of max_i max_j per
    row, dominate the rounding of F)."""
    planes, bits, _, _ = SCHEMES[name]
    rng = np.random.default_rng(seed)
    n, c = 24, 3
    Y = rng.standard_normal((n, c)) * np.exp2(rng.integers(-spread, spread + 1, (n, c))) * np.array([1.0, 1e-5, 3e4])
    G = digit_gram(Y, planes, bits)
    for i in range(c):
        for j in range(i, c):
            exact = sum(Fraction(float(Y[r, i])) * Fraction(float(Y[r, j])) for r in range(n))
            err = abs(G[i][j] - exact)
            ni2 = sum(Fraction(float(v)) ** 2 for v in Y[:, i])
            nj2 = sum(Fraction(float(v)) ** 2 for v in Y[:, j])
            assert err ** 2 <= Fraction(2) ** -106 * ni2 * nj2
            mi = max(abs(Fraction(float(v))) for v in Y[:, i])
            mj = max(abs(Fraction(float(v))) for v in Y[:, j])
            assert err <= n * Fraction(2) ** -56 * mi * mj


@scheme
def test_digit_gram_componentwise_caveat(name):
    """Componentwise the scheme is not binary64's equal: an entry whose
    products all lie far below the two columns' largest values keeps only
    the absolute accuracy set by those maxima.  Here G_01 sums products near
    2^-60 while each column holds a 1.0 in a row where the other is zero."""
    Y = np.zeros((6, 2))
    Y[0, 0] = 1.0
    Y[1, 1] = 1.0
    Y[2:, 0] = np.array([1.3, -0.7, 1.1, 0.9]) * 2.0 ** -30
    Y[2:, 1] = np.array([0.6, 1.7, -1.2, 0.8]) * 2.0 ** -30
    G = digit_gram(Y, *SCHEMES[name][:2])
    exact = sum(Fraction(float(Y[r, 0])) * Fraction(float(Y[r, 1])) for r in range(6))
    absum = sum(abs(Fraction(float(Y[r, 0])) * Fraction(float(Y[r, 1]))) for r in range(6))
    err = abs(G[0][1] - exact)
    assert err > 6 * Fraction(2) ** -53 * absum   # beyond binary64's componentwise bound
    assert err <= Fraction(2) ** -53              # yet far below 2^-53 max_0 max_1 = 2^-53


@scheme
def test_digit_gram_exact_on_integers(name):
    """Integer entries below 2^16 have exact digits and exact products: the
    digit Gram is the integer Gram."""
    rng = np.random.default_rng(9)
    Y = rng.integers(-(2 ** 15), 2 ** 15, (30, 3)).astype(np.float64)
    G = digit_gram(Y, *SCHEMES[name][:2])
    Gi = Y.astype(np.int64).T @ Y.astype(np.int64)
    for i in range(3):
        for j in range(3):
            assert G[i][j] == Gi[i, j]
