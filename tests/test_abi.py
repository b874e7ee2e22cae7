"""Host-side checks of the C ABI (no GPU needed): the library builds for sm_103a, exports every
entry point declared in include/ozg.h, and rejects invalid BLAS arguments with xerbla
numbering before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "ozg.h")).read()
    return re.findall(r"^(?:int|const char\*)\s+(ozg_\w+)\s*\(", txt, re.M)


@pytest.fixture(scope="module")
def lib():
    from paper_2503_22875_gb300 import build, ozg
    build.build()
    return ozg.load()


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_strerror_codes(lib):
    from paper_2503_22875_gb300 import ozg
    assert "success" in ozg.strerror(0)
    assert "argument" in ozg.strerror(-8)
    assert "wait" in ozg.strerror(3)


@pytest.mark.parametrize("args,code", [
    (("X", "N", 4, 4, 4, 4, 4, 4, 7), -1),
    (("N", "Q", 4, 4, 4, 4, 4, 4, 7), -2),
    (("N", "N", -1, 4, 4, 4, 4, 4, 7), -3),
    (("N", "N", 4, -1, 4, 4, 4, 4, 7), -4),
    (("N", "N", 4, 4, -1, 4, 4, 4, 7), -5),
    (("N", "N", 4, 4, 4, 3, 4, 4, 7), -8),
    (("T", "N", 4, 4, 5, 4, 5, 4, 7), -8),     # op(A) = A^T: A is k x m, lda >= k
    (("N", "N", 4, 4, 4, 4, 3, 4, 7), -10),
    (("N", "T", 4, 6, 4, 4, 4, 4, 7), -10),    # B is n x k, ldb >= n
    (("N", "N", 4, 4, 4, 4, 4, 3, 7), -13),
    (("N", "N", 4, 4, 4, 4, 4, 4, 0), 5),      # 0 = automatic slice count: valid; null context
    (("N", "N", 4, 4, 4, 4, 4, 4, 19), -14),
    (("N", "N", 4, 4, 4, 4, 4, 4, -2), -14),
])
def test_dgemm_argument_errors(lib, args, code):
    ta, tb, m, n, k, lda, ldb, ldc, s = args
    rc = lib.ozg_dgemm(None, ta.encode(), tb.encode(), m, n, k, 1.0, None, lda, None, ldb, 0.0, None, ldc, s, None)
    assert rc == code


def test_zgemm_accepts_conjugate_and_checks_args(lib):
    al = (ctypes.c_double * 2)(1.0, 0.0)
    rc = lib.ozg_zgemm(None, b"C", b"C", 4, 4, 4, al, None, 4, None, 4, al, None, 4, 7, None)
    assert rc == 5  # arguments valid, null context -> OZG_ERR_INVALID
    rc = lib.ozg_zgemm(None, b"C", b"N", 4, 4, 6, al, None, 5, None, 6, al, None, 4, 7, None)
    assert rc == -8


def test_null_context(lib):
    assert lib.ozg_sync(None) == 5
    assert lib.ozg_destroy(None) == 0


def test_blas_shim_exports_and_mode_parsing():
    from paper_2503_22875_gb300 import build
    build.build()
    shim = ctypes.CDLL(build.SHIM_LIB)
    txt = open(os.path.join(ROOT, "include", "ozg_blas.h")).read()
    names = re.findall(r"^(?:void|int|long long)\s+(\w+)\s*\(", txt, re.M)
    assert {"dgemm_", "zgemm_", "ozg_blas_parse_mode"} <= set(names)
    for n in names:
        assert hasattr(shim, n), n
    shim.ozg_blas_parse_mode.argtypes = [ctypes.c_char_p]
    cases = {b"dgemm": -1, b"fp64_int8_3": 3, b"fp64_int8_18": 18, b"fp64_int8_7": 7, b"fp64_int8_19": 0,
             b"fp64_int8_0": 0, b"fp64_int8_": 0, b"fp64_int8_x": 0, b"int8_7": 0, b"": 0, b"DGEMM": 0}
    for s, v in cases.items():
        assert shim.ozg_blas_parse_mode(s) == v, s
    shim.ozg_blas_parse_strategy.argtypes = [ctypes.c_char_p]
    for s, v in {b"copy": 0, b"coherent": 1, b"migrate": 2, b"": -1, b"COPY": -1, b"uma": -1}.items():
        assert shim.ozg_blas_parse_strategy(s) == v, s
    shim.ozg_blas_set_strategy.argtypes = [ctypes.c_int]
    assert shim.ozg_blas_set_strategy(3) == -1 and shim.ozg_blas_set_strategy(-1) == -1


@pytest.mark.parametrize("args,code", [
    (("N", "N", 4, 4, 4, 4, 4, 4, 2, 2), 5),    # valid arguments, null context
    (("X", "N", 4, 4, 4, 4, 4, 4, 2, 2), -1),
    (("N", "N", 4, 4, 4, 3, 4, 4, 2, 2), -8),
    (("N", "T", 4, 6, 4, 4, 4, 4, 2, 2), -10),
    (("N", "N", 4, 4, 4, 4, 4, 3, 2, 2), -13),
    (("N", "N", 4, 4, 4, 4, 4, 4, 0, 2), -14),  # row_blocks
    (("N", "N", 4, 4, 4, 4, 4, 4, 2, 0), -15),  # col_blocks
])
def test_regions_argument_errors(lib, args, code):
    ta, tb, m, n, k, lda, ldb, ldc, rb, cb = args
    rc = lib.ozg_dgemm_regions(None, ta.encode(), tb.encode(), m, n, k, 1.0, None, lda, None, ldb, 0.0, None, ldc,
                               rb, cb, None)
    assert rc == code


@pytest.mark.parametrize("args,code", [
    (("C", "T", 4, 4, 4, 4, 4, 4, 7), 5),       # valid arguments, null context
    (("Q", "N", 4, 4, 4, 4, 4, 4, 7), -1),
    (("N", "N", 4, -1, 4, 4, 4, 4, 7), -4),
    (("C", "N", 4, 4, 6, 5, 6, 4, 7), -8),      # op(A) = A^H: A is k x m, lda >= k
    (("N", "N", 4, 4, 4, 4, 4, 2, 7), -13),
    (("N", "N", 4, 4, 4, 4, 4, 4, 0), -14),     # the selector is not used for 3M
    (("N", "N", 4, 4, 4, 4, 4, 4, -1), 5),      # native FP64 is valid
])
def test_zgemm3m_argument_errors(lib, args, code):
    ta, tb, m, n, k, lda, ldb, ldc, s = args
    al = (ctypes.c_double * 2)(1.0, 0.0)
    rc = lib.ozg_zgemm3m(None, ta.encode(), tb.encode(), m, n, k, al, None, lda, None, ldb, al, None, ldc, s, None)
    assert rc == code
