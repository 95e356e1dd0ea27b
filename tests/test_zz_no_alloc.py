"""sscg_gram_noalloc against sscg_gram, through the C ABI (collected last).

sscg_gram_noalloc serves callers that may not allocate device memory inside a
library call (fixed device-memory budgets, hosts whose own allocator owns the
device); it keeps its block partials in a fixed array inside the library.
Its result must match sscg_gram's within the Gram tolerance of the parity
tests (1e-13 relative to sqrt(G_ii G_jj)), on two calls in a row, run alone
in a fresh process or after every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_04081_gb300 import sscg
    return sscg.load_library()


def _columns(n, ncols, seed):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((n, ncols)) * np.logspace(0, 4, ncols)[None, :]
    ld = n + 7
    Yd = torch.zeros(ld * ncols, dtype=torch.float64, device="cuda")
    Yd.reshape(ncols, ld)[:, :n] = torch.tensor(Y.T.copy(), device="cuda")
    return Y, Yd, ld


def _gram(fn, Yd, n, ld, ncols):
    G = torch.full((ncols * ncols,), float("nan"), dtype=torch.float64, device="cuda")
    rc = fn(ctypes.c_void_p(Yd.data_ptr()), n, ld, ncols, ctypes.c_void_p(G.data_ptr()), None)
    assert rc == 0
    torch.cuda.synchronize()
    return G.reshape(ncols, ncols).cpu().numpy()


def test_noalloc_gram_matches_gram_on_two_calls(lib):
    # two calls in a row with different shapes: the second must not see the
    # first call's partial sums
    for n, ncols, seed in ((200003, 33, 1), (1000, 5, 2)):
        Y, Yd, ld = _columns(n, ncols, seed)
        G_ref = _gram(lib.sscg_gram, Yd, n, ld, ncols)
        G_na = _gram(lib.sscg_gram_noalloc, Yd, n, ld, ncols)
        d = np.sqrt(np.outer(np.diag(G_ref), np.diag(G_ref)))
        assert np.all(np.isfinite(G_na))
        assert np.max(np.abs(G_na - G_ref) / d) <= 1e-13
        assert np.max(np.abs(G_na - Y.T @ Y) / d) <= 1e-13


def test_noalloc_gram_rejects_too_many_columns(lib):
    Y, Yd, ld = _columns(100, 3, 3)
    G = torch.zeros(34 * 34, dtype=torch.float64, device="cuda")
    rc = lib.sscg_gram_noalloc(ctypes.c_void_p(Yd.data_ptr()), 100, ld, 34, ctypes.c_void_p(G.data_ptr()), None)
    assert rc == -1   # SSCG_ERR_INVALID_ARG: the scratch holds partials for at most 33 columns
