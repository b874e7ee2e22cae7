"""The dgemm_/zgemm_ interposition library (host buffers, synchronous) against
the oracle, and its interposition over a CPU BLAS with LD_PRELOAD."""
import ctypes
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle
from paper_2503_22875_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U = 2.0 ** -53
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def shim():
    from paper_2503_22875_gb300 import build
    build.build()
    lib = ctypes.CDLL(build.SHIM_LIB)
    lib.ozg_blas_set_mode.argtypes = [ctypes.c_int]
    lib.ozg_blas_offloaded_calls.restype = ctypes.c_longlong
    lib.ozg_blas_set_strategy.argtypes = [ctypes.c_int]
    lib.ozg_blas_migrated_bytes.restype = ctypes.c_longlong
    return lib


def call(lib, name, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc):
    i = ctypes.c_int
    cplx = name == "zgemm_"
    if cplx:
        al = (ctypes.c_double * 2)(alpha.real, alpha.imag)
        be = (ctypes.c_double * 2)(beta.real, beta.imag)
    else:
        al, be = ctypes.c_double(alpha), ctypes.c_double(beta)
    getattr(lib, name)(ta.encode(), tb.encode(), ctypes.byref(i(m)), ctypes.byref(i(n)), ctypes.byref(i(k)),
                       ctypes.byref(al), A.ctypes.data_as(ctypes.c_void_p), ctypes.byref(i(lda)),
                       B.ctypes.data_as(ctypes.c_void_p), ctypes.byref(i(ldb)), ctypes.byref(be),
                       C.ctypes.data_as(ctypes.c_void_p), ctypes.byref(i(ldc)), ctypes.c_size_t(1),
                       ctypes.c_size_t(1))


def test_shim_dgemm_emulated(shim):
    assert shim.ozg_blas_set_mode(7) == 0
    m, n, k, s = 130, 70, 300, 7
    A, B = workloads.wide_exponent_pair(m, n, k, 1.0, seed=201)
    At = np.asfortranarray(A.T)  # op(A) = At^T
    ldc = m + 4
    C0 = np.asfortranarray(workloads.rng(202).uniform(-1, 1, (ldc, n)))
    C = C0.copy(order="F")
    before = shim.ozg_blas_offloaded_calls()
    call(shim, "dgemm_", "T", "N", m, n, k, 0.5, At, k, B, k, -2.0, C, ldc)
    assert shim.ozg_blas_offloaded_calls() == before + 1
    E = oracle.dgemm_emu(At, B, s, "T", "N", 0.5, -2.0, np.asfortranarray(C0[:m]))
    AB = np.abs(A) @ np.abs(B)
    tol = 4 * (s + 2) * U * 0.5 * AB + 2 * U * np.abs(E) + 4 * U * np.abs(C0[:m])
    assert (np.abs(C[:m] - E) <= tol).all()
    assert np.array_equal(C[m:], C0[m:])  # rows m..ldc-1 untouched


def test_shim_zgemm_and_native_mode(shim):
    m, n, k = 40, 50, 60
    A = workloads.wide_exponent((k, m), 0.5, workloads.rng(203)) + 1j * workloads.wide_exponent((k, m), 0.5, workloads.rng(204))
    B = workloads.wide_exponent((k, n), 0.5, workloads.rng(205)) + 1j * workloads.wide_exponent((k, n), 0.5, workloads.rng(206))
    A, B = np.asfortranarray(A), np.asfortranarray(B)
    assert shim.ozg_blas_set_mode(8) == 0
    C = np.zeros((m, n), dtype=np.complex128, order="F")
    call(shim, "zgemm_", "C", "N", m, n, k, 1.0 + 0j, A, k, B, k, 0j, C, m)
    E = oracle.zgemm_emu(A, B, 8, "C", "N")
    scale = (np.abs(A.real) + np.abs(A.imag)).T @ (np.abs(B.real) + np.abs(B.imag))
    assert (np.abs(C - E) <= 8 * 10 * U * scale + 4 * U * np.abs(E)).all()
    assert shim.ozg_blas_set_mode(-1) == 0  # "dgemm" mode: native FP64
    Cn = np.zeros((m, n), dtype=np.complex128, order="F")
    call(shim, "zgemm_", "C", "N", m, n, k, 1.0 + 0j, A, k, B, k, 0j, Cn, m)
    np.testing.assert_allclose(Cn, A.conj().T @ B, rtol=0, atol=(k + 2) * 4 * U * scale.max())
    assert shim.ozg_blas_set_mode(7) == 0


def test_shim_interposes_with_ld_preload(shim, tmp_path):
    from paper_2503_22875_gb300 import build
    # a stand-in CPU BLAS whose dgemm_ writes a sentinel, and a program that calls dgemm_
    (tmp_path / "fake.c").write_text(textwrap.dedent("""
        #include <stddef.h>
        void dgemm_(const char* ta, const char* tb, const int* m, const int* n, const int* k, const double* al,
                    const double* A, const int* lda, const double* B, const int* ldb, const double* be, double* C,
                    const int* ldc, size_t l1, size_t l2) {
          for (int j = 0; j < *n; ++j) for (int i = 0; i < *m; ++i) C[i + j * *ldc] = 42.0;
        }"""))
    (tmp_path / "prog.c").write_text(textwrap.dedent("""
        #include <stdio.h>
        #include <stddef.h>
        void dgemm_(const char*, const char*, const int*, const int*, const int*, const double*, const double*,
                    const int*, const double*, const int*, const double*, double*, const int*, size_t, size_t);
        int main(void) {
          int m = 64, n = 64, k = 64;
          static double A[64 * 64], B[64 * 64], C[64 * 64];
          for (int i = 0; i < 64 * 64; ++i) { A[i] = (i % 7) - 3; B[i] = (i % 5) - 2; }
          double one = 1.0, zero = 0.0;
          dgemm_("N", "N", &m, &n, &k, &one, A, &m, B, &k, &zero, C, &m, 1, 1);
          double ref = 0.0;
          for (int l = 0; l < 64; ++l) ref += A[0 + l * 64] * B[l + 0 * 64];
          printf("%.17g %.17g\\n", C[0], ref);
          return 0;
        }"""))
    subprocess.check_call(["gcc", "-shared", "-fPIC", "-o", str(tmp_path / "libfakeblas.so"), str(tmp_path / "fake.c")])
    subprocess.check_call(["gcc", "-o", str(tmp_path / "prog"), str(tmp_path / "prog.c"), "-L", str(tmp_path),
                           "-lfakeblas", f"-Wl,-rpath,{tmp_path}"])
    env = dict(os.environ, OZG_COMPUTE_MODE="fp64_int8_7")
    plain = subprocess.run([str(tmp_path / "prog")], capture_output=True, text=True, env=env, check=True)
    assert plain.stdout.split()[0] == "42"
    env["LD_PRELOAD"] = build.SHIM_LIB
    out = subprocess.run([str(tmp_path / "prog")], capture_output=True, text=True, env=env, check=True)
    got, ref = map(float, out.stdout.split())
    assert got == ref  # small integers: the emulation is exact
    env["OZG_OFFLOAD_MIN_MNK"] = str(10 ** 9)  # below the threshold -> the next (CPU) BLAS
    out = subprocess.run([str(tmp_path / "prog")], capture_output=True, text=True, env=env, check=True)
    assert out.stdout.split()[0] == "42"


STRATEGIES = {0: "copy", 1: "coherent", 2: "migrate"}


def in_place_supported(shim, strategy):
    assert shim.ozg_blas_set_strategy(strategy) == 0
    # the device check runs at the first GPU use: make one tiny call, then read the strategy
    C = np.zeros((1, 1), order="F")
    one = np.ones((1, 1), order="F")
    call(shim, "dgemm_", "N", "N", 1, 1, 1, 1.0, one, 1, one, 1, 0.0, C, 1)
    return shim.ozg_blas_get_strategy() == strategy


def test_shim_data_strategies_same_bits(shim):
    """The three data strategies (DMA copies, coherent in-place access, migration on first
    use) give the same bits: a real call with beta != 0 and padding rows (left untouched), equal
    to the oracle's definition, and a complex conjugate-transpose call."""
    assert shim.ozg_blas_set_mode(7) == 0
    m, n, k = 130, 70, 300
    A, B = workloads.wide_exponent_pair(m, n, k, 1.0, seed=211)
    ldc = m + 3
    C0 = np.asfortranarray(workloads.rng(212).uniform(-1, 1, (ldc, n)))
    mz, nz, kz = 45, 38, 77
    g = workloads.rng(213)
    Az = np.asfortranarray(workloads.wide_exponent((kz, mz), 0.5, g) + 1j * workloads.wide_exponent((kz, mz), 0.5, g))
    Bz = np.asfortranarray(workloads.wide_exponent((kz, nz), 0.5, g) + 1j * workloads.wide_exponent((kz, nz), 0.5, g))
    Z0 = np.asfortranarray(g.normal(size=(mz, nz)) + 1j * g.normal(size=(mz, nz)))
    res = {}
    try:
        for st in STRATEGIES:
            if st and not in_place_supported(shim, st):
                pytest.skip(f"this GPU cannot access pageable host memory ({STRATEGIES[st]} falls back)")
            assert shim.ozg_blas_set_strategy(st) == 0
            C = C0.copy(order="F")
            call(shim, "dgemm_", "N", "N", m, n, k, 0.75, A, m, B, k, -0.5, C, ldc)
            Z = Z0.copy(order="F")
            call(shim, "zgemm_", "C", "N", mz, nz, kz, 0.5 - 1j, Az, kz, Bz, kz, 0.25 + 0.5j, Z, mz)
            assert shim.ozg_blas_get_strategy() == st
            res[st] = (C, Z)
    finally:
        shim.ozg_blas_set_strategy(0)
    E = oracle.dgemm_emu(A, B, 7, "N", "N", 0.75, -0.5, np.asfortranarray(C0[:m]))
    assert np.array_equal(res[0][0][:m], E)
    assert np.array_equal(res[0][0][m:], C0[m:])
    for st in (1, 2):
        assert np.array_equal(res[st][0], res[0][0]), STRATEGIES[st]
        assert np.array_equal(res[st][1], res[0][1]), STRATEGIES[st]


def test_shim_migrate_first_use_and_coherence(shim):
    """Migration on first use moves the arrays' pages once: a second call on the same arrays
    moves nothing. After the CPU rewrites A in place (coherent access to pages now in GPU
    memory), the next call sees the new values, and moves nothing either."""
    assert shim.ozg_blas_set_mode(7) == 0
    try:
        if not in_place_supported(shim, 2):
            pytest.skip("this GPU cannot migrate pageable host memory (migrate falls back)")
        m, n, k = 256, 192, 320
        A, B = workloads.wide_exponent_pair(m, n, k, 2.0, seed=221)
        C = np.zeros((m, n), order="F")
        b0 = shim.ozg_blas_migrated_bytes()
        call(shim, "dgemm_", "N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m)
        b1 = shim.ozg_blas_migrated_bytes()
        assert b1 - b0 >= A.nbytes + B.nbytes + C.nbytes - 3 * 2 * 65536  # page-rounded spans
        assert np.array_equal(C, oracle.dgemm_emu(A, B, 7, "N", "N"))
        call(shim, "dgemm_", "N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m)
        assert shim.ozg_blas_migrated_bytes() == b1
        A *= 2.0  # the CPU writes the moved pages in place
        A[3, 5] = -7.25
        call(shim, "dgemm_", "N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m)
        assert shim.ozg_blas_migrated_bytes() == b1
        assert np.array_equal(C, oracle.dgemm_emu(A, B, 7, "N", "N"))
    finally:
        shim.ozg_blas_set_strategy(0)
