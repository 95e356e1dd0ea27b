"""The C-ABI library loads and exports every symbol include/sscg.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sscg.h")
LIB = os.path.join(ROOT, "paper_1908_04081_gb300", "libsscg.so")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(sscg_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_1908_04081_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("sscg_create_csr", "sscg_create_stencil", "sscg_solve", "sscg_solve_hscg",
                 "sscg_ritz", "sscg_destroy", "sscg_strerror", "sscg_gram", "sscg_kappa"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    lib.sscg_strerror.restype = ctypes.c_char_p
    assert lib.sscg_strerror(0) == b"ok"
    assert b"invalid" in lib.sscg_strerror(-1)
    lib.sscg_version.restype = ctypes.c_char_p
    assert b"sscg" in lib.sscg_version()


def test_binding_rejects_unknown_options(lib):
    from paper_1908_04081_gb300 import sscg
    with pytest.raises(sscg.SscgError):
        sscg.sscg_opts_default(mpk_fp64_per_16=8)   # misspelt: not a field of sscg_opts
    assert sscg.sscg_opts_default(mpk_fp64_per16=8).mpk_fp64_per16 == 8


def test_binding_defaults(lib):
    from paper_1908_04081_gb300 import sscg
    o = sscg.sscg_opts_default()
    assert o.inner_conv_check == 1 and o.eps == 2.0 ** -53 and o.kappa_cut == 2.0 ** -44
    o2 = sscg.sscg_opts_default(c_mode="one", variant="fixed")
    assert o2.c_mode == 2 and o2.variant == 1
    assert o.gram_mode == 0  # the method as written
    assert sscg.sscg_opts_default(gram_mode="digits").gram_mode == 2
    assert sscg.sscg_opts_default(gram_mode="binary32_pair").gram_mode == 1
    assert sscg.sscg_opts_default(gram_mode="digits_tcgen05").gram_mode == 3
    # the FP64/integer split of the stencil matrix-powers level: -1 (library default) .. 16
    assert sscg.sscg_opts_default().mpk_fp64_per16 == -1
    assert L_opts_rejects_split(sscg)
    # the same for the recovery's split
    assert sscg.sscg_opts_default().rec_fp64_per16 == -1
    assert L_opts_rejects_split(sscg, "rec_fp64_per16")
    # exact Ritz values (0 = Algorithms 3-4, 1 = eigenvalues of T_m): other values rejected
    assert sscg.sscg_opts_default().ritz_exact == 0
    L = sscg.load_library()
    o = sscg.sscg_opts_default(ritz_exact=2)
    assert L.sscg_solve(ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), 1e-10, 8, 2,
                        ctypes.byref(o), None) == -1


def test_invalid_arguments_rejected_without_gpu(lib):
    from paper_1908_04081_gb300 import sscg
    L = sscg.load_library()
    h = ctypes.c_void_p()
    assert L.sscg_create_csr(ctypes.byref(h), 0, 0, None, None, None, 0, None) == -1
    assert L.sscg_solve(None, None, None, 1e-10, 8, 2, None, None) == -1
    assert L.sscg_leja(0, None) == -1
    # Gram product arithmetic outside 0..3 is rejected before any pointer is used
    fake = ctypes.c_void_p(16)
    for mode in (-1, 4):
        assert L.sscg_gram_ex(fake, ctypes.c_int64(10), ctypes.c_int64(10), 3, fake, mode, None) == -1
    # the recovery step: sizes and split checked before any pointer is used
    coef = (ctypes.c_double * 9)()
    n10 = ctypes.c_int64(10)
    assert L.sscg_recombine(fake, ctypes.c_int64(0), n10, 3, coef, fake, -1, None) == -1
    assert L.sscg_recombine(fake, n10, ctypes.c_int64(9), 3, coef, fake, -1, None) == -1
    assert L.sscg_recombine(fake, n10, n10, 34, coef, fake, -1, None) == -1
    assert L.sscg_recombine(fake, n10, n10, 3, coef, fake, 17, None) == -1
    assert L.sscg_recombine(fake, n10, n10, 3, coef, fake, -2, None) == -1
    # the comparator's and the SpMV's split: -1..16
    for split in (-2, 17):
        assert L.sscg_solve_hscg_ex(fake, fake, fake, 1e-10, 0, split, None) == -1
        assert L.sscg_spmv_ex(fake, fake, fake, split) == -1
    assert L.sscg_solve_hscg_ex(fake, fake, fake, 0.0, 0, 16, None) == -1
    # the batch autotuner with the Gram as a candidate dimension: arguments checked first
    assert L.sscg_autotune_batch_ex(None, 0, None, None, 1e-10, None, 2, None, None, None, 0, 1, None, None,
                                    None) == -1


def L_opts_rejects_split(sscg, field="mpk_fp64_per16"):
    """A split outside -1..16 is rejected (before any GPU work)."""
    L = sscg.load_library()
    o = sscg.sscg_opts_default(**{field: 17})
    return L.sscg_solve(ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), 1e-10, 8, 2,
                        ctypes.byref(o), None) == -1
