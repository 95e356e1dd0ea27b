"""GPU parity of the recovery x += Y x', r = Y r', p = Y p' (eq. coords,
Algorithm 5) through sscg_recombine, for every split of its rows between
binary64 FMA chains and exact integer dot products.

Expected values are exact: on sampled rows every product and sum is taken in
rational arithmetic (fractions.Fraction), so each form is held to its own
bound -
- integer rows: within m (1 + 2^-5) 2^-54 of the largest |term| before the
  one final rounding (half an ulp of the exact sum), m = nc + 1 terms
  (x enters as x * 1);
- FMA rows: within m 2^-53 sum|terms| (the recursive-summation bound), plus
  half an ulp for x's addition;
and a split row by row equals, bit for bit, the run of the form its row group
takes (groups of 32 rows; group g is summed by FMAs when (5 g) mod 16 < 5 for
the split 5).  Non-finite inputs and sums outside the binary64 range fall back
to the FMA chains.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_04081_gb300 as p
    p.load_library()
    return p


def run(pkg, Y, x, coef, nc, split):
    n, ld = x.size, Y.shape[0]
    Yd = torch.tensor(Y.T.copy().ravel(), dtype=torch.float64, device="cuda")   # column major, leading dim ld
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    pkg.sscg.sscg_recombine(Yd, n, ld, nc, coef, xd, split)
    torch.cuda.synchronize()
    Yo = Yd.cpu().numpy().reshape(-1, ld)
    return xd.cpu().numpy(), Yo[1, :n].copy(), Yo[0, :n].copy()   # x, r (column 1), p (column 0)


def exact_rows(Y, x, coef, nc, rows):
    """Exact x + Y x', Y r', Y p' and the largest |term| and sum|terms| of each."""
    cx, cr, cp = (coef[k * nc:(k + 1) * nc] for k in range(3))
    out = []
    for i in rows:
        ys = [Fraction(float(Y[i, c])) for c in range(nc)]
        res = []
        for k, cc in enumerate((cx, cr, cp)):
            terms = [y * Fraction(float(c)) for y, c in zip(ys, cc)]
            if k == 0:
                terms.append(Fraction(float(x[i])))
            res.append((sum(terms), max(abs(t) for t in terms), sum(abs(t) for t in terms), len(terms)))
        out.append(res)
    return out


def problem(n, ld, nc, seed, spread=0):
    """Y with column and row scales 2^U(-spread, spread); coefficients alternating
    in sign and falling like a coordinate vector (10^-c), x of unit size."""
    rng = np.random.default_rng(seed)
    Y = np.zeros((ld, max(nc, 2)))          # the recovery writes columns 0 and 1
    Y[:n, :nc] = rng.standard_normal((n, nc))
    if spread:
        Y[:n, :nc] *= np.exp2(rng.integers(-spread, spread + 1, (n, 1)))
        Y[:n, :nc] *= np.exp2(rng.integers(-spread, spread + 1, (1, nc)))
    c = rng.standard_normal(3 * nc) * np.tile(10.0 ** -np.arange(nc) * (-1.0) ** np.arange(nc), 3)
    x = rng.standard_normal(n)
    return Y, x, c


def fma_group(i, split):
    g = i >> 5
    return ((g * split) & 15) < split


@pytest.mark.parametrize("n,nc,spread", [(1, 1, 0), (33, 3, 0), (1000, 17, 0), (70001, 33, 0), (20000, 25, 300),
                                         (5000, 33, 40)])
def test_recombine_each_form_within_its_bound(pkg, n, nc, spread):
    ld = n + 7
    Y, x, coef = problem(n, ld, nc, seed=n + nc, spread=spread)
    res = {s: run(pkg, Y, x, coef, nc, s) for s in (0, 16, 5)}
    rng = np.random.default_rng(7)
    rows = np.unique(np.concatenate([rng.integers(0, n, min(n, 300)), [0, n - 1]]))
    ex = exact_rows(Y, x, coef, nc, rows)
    for s, tol_kind in ((0, "int"), (16, "fma")):
        outs = res[s]
        for ri, i in enumerate(rows):
            for k in range(3):
                val, tmax, tsum, m = ex[ri][k]
                got = Fraction(float(outs[k][i]))
                half_ulp = Fraction(math.ulp(float(val))) / 2 if val != 0 else Fraction(0)
                if tol_kind == "int":
                    bound = m * Fraction(33, 32) * tmax / 2 ** 54 + 2 * half_ulp
                else:
                    bound = Fraction(101, 100) * m * tsum / 2 ** 53 + 2 * half_ulp
                assert abs(got - val) <= bound, (s, k, i, float(got), float(val), float(bound))
    # the mixed split equals the form of each row's group, bit for bit
    grp = np.array([fma_group(i, 5) for i in range(n)])
    for k in range(3):
        want = np.where(grp, res[16][k], res[0][k])
        assert np.array_equal(res[5][k], want), k


def test_recombine_nonfinite_and_out_of_range_rows_take_the_fma_chains(pkg):
    n, nc = 4096, 9
    ld = n
    Y, x, coef = problem(n, ld, nc, seed=3)
    Y[10, 4] = np.nan
    Y[77, 0] = np.inf
    Y[500, :] = 1e308              # with the first coefficients 10: sums past the binary64 range
    x[500] = 0.0
    Y[900, :] = 1e-310             # subnormal results
    x[900] = 0.0
    Y[1300, 2] = -np.inf
    x[2000] = np.nan
    coef[0] = coef[nc] = coef[2 * nc] = 10.0
    ref = run(pkg, Y, x, coef, nc, 16)
    got = run(pkg, Y, x, coef, nc, 0)
    for k in range(3):
        a, b = got[k], ref[k]
        assert np.array_equal(np.isnan(a), np.isnan(b)), k
        fin = np.isfinite(b)
        assert np.array_equal(np.isinf(a), np.isinf(b)) and np.array_equal(a[np.isinf(a)], b[np.isinf(b)]), k
        for i in (10, 77, 500, 900, 1300, 2000):
            assert (np.isnan(a[i]) and np.isnan(b[i])) or a[i] == b[i], (k, i, a[i], b[i])
        # every other row is finite and close
        assert np.all(np.abs(a[fin] - b[fin]) <= 1e-13 * (1 + np.abs(b[fin]))), k


def test_recombine_coefficients_nonfinite_whole_call_on_fma(pkg):
    n, nc = 3000, 5
    Y, x, coef = problem(n, n, nc, seed=11)
    coef[3] = np.inf
    a = run(pkg, Y, x, coef, nc, 0)
    b = run(pkg, Y, x, coef, nc, 16)
    for k in range(3):
        assert np.array_equal(a[k], b[k], equal_nan=True), k


def test_recombine_integer_sum_of_integers_is_exact(pkg):
    """Integer Y and coefficients: every product and sum is an integer below
    2^53, so both forms give the exact result."""
    n, nc = 10000, 33
    rng = np.random.default_rng(5)
    Y = rng.integers(-2 ** 20, 2 ** 20, (n, nc)).astype(np.float64)
    coef = rng.integers(-2 ** 20, 2 ** 20, 3 * nc).astype(np.float64)
    x = rng.integers(-2 ** 40, 2 ** 40, n).astype(np.float64)
    Yi, ci, xi = Y.astype(object), coef.astype(object), x.astype(object)
    want = [xi + Yi @ ci[:nc], Yi @ ci[nc:2 * nc], Yi @ ci[2 * nc:]]
    for s in (0, 16):
        got = run(pkg, Y, x, coef, nc, s)
        for k in range(3):
            assert all(int(g) == w for g, w in zip(got[k], want[k])), (s, k)
