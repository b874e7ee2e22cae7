"""Pins for the CPU oracle (no GPU).  Each test ties one oracle function to something other
than itself: exact rational arithmetic, brute force with Python integers, closed forms,
invariants of the splitting, or the a priori error bound derived for the method (Sec. 2.2:
the Ozaki scheme's split into low-precision slices with high-precision accumulation)."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

U = 2.0 ** -53


def frac_matmul(A, B):
    m, k = A.shape
    n = B.shape[1]
    return [[sum(Fraction(float(A[i, l])) * Fraction(float(B[l, j])) for l in range(k)) for j in range(n)]
            for i in range(m)]


# --------------------------------------------------------------------------- double-double
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_dd_matches_exact_rationals(seed):
    rng = np.random.default_rng(seed)
    m, k, n = 3, 8, 4
    A = rng.uniform(-1, 1, (m, k)) * np.exp(rng.normal(0, 8, (m, k)))
    B = rng.uniform(-1, 1, (k, n)) * np.exp(rng.normal(0, 8, (k, n)))
    hi, lo = oracle.dgemm_dd(A, B)
    ex = frac_matmul(A, B)
    absAB = np.abs(A) @ np.abs(B)
    for i in range(m):
        for j in range(n):
            err = abs(Fraction(hi[i, j]) + Fraction(lo[i, j]) - ex[i][j])
            assert err <= Fraction(4 * k) * Fraction(U) ** 2 * Fraction(absAB[i, j] * 1.01)
            assert hi[i, j] == float(Fraction(hi[i, j]) + Fraction(lo[i, j]))  # normalised pair


def test_dd_alpha_beta_exact():
    A = np.array([[1.0 + 2 ** -40, 3.0]])
    B = np.array([[1.0 - 2 ** -40], [2.0 ** -60]])
    C0 = np.array([[0.25]])
    hi, lo = oracle.dgemm_dd(A, B, alpha=3.0, beta=-0.5, C=C0)
    ex = Fraction(3) * (Fraction(A[0, 0]) * Fraction(B[0, 0]) + Fraction(3.0) * Fraction(B[1, 0])) - Fraction(1, 8)
    assert abs(Fraction(hi[0, 0]) + Fraction(lo[0, 0]) - ex) <= abs(ex) * Fraction(2) ** -100


def test_naive_within_gamma_k():
    rng = np.random.default_rng(3)
    m, k, n = 5, 40, 6
    A = rng.normal(size=(m, k))
    B = rng.normal(size=(k, n))
    C = oracle.dgemm_naive(A, B)
    ex = frac_matmul(A, B)
    absAB = np.abs(A) @ np.abs(B)
    gk = k * U / (1 - k * U)
    for i in range(m):
        for j in range(n):
            assert abs(Fraction(C[i, j]) - ex[i][j]) <= Fraction(gk * absAB[i, j] * 1.0001)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_naive_transposes_and_beta(ta, tb):
    rng = np.random.default_rng(4)
    m, k, n = 7, 5, 3
    A = rng.normal(size=(m, k) if ta == "N" else (k, m))
    B = rng.normal(size=(k, n) if tb == "N" else (n, k))
    C0 = rng.normal(size=(m, n))
    opA = A if ta == "N" else A.T
    opB = B if tb == "N" else B.T
    C = oracle.dgemm_naive(A, B, ta, tb, alpha=2.0, beta=-1.5, C=C0)
    np.testing.assert_allclose(C, 2.0 * opA @ opB - 1.5 * C0, rtol=1e-13, atol=1e-13)
    # beta == 0: NaN in C is never read
    Cn = np.full((m, n), np.nan)
    C = oracle.dgemm_naive(A, B, ta, tb, alpha=1.0, beta=0.0, C=Cn)
    assert np.isfinite(C).all()


# --------------------------------------------------------------------------- splitter
def reconstruct(e, D, s=None):
    s = D.shape[0] if s is None else s
    rows, k = D.shape[1], D.shape[2]
    out = []
    for i in range(rows):
        row = []
        for l in range(k):
            v = sum(Fraction(int(D[t, i, l])) * Fraction(1, 128 ** (t + 1)) for t in range(s))
            row.append(v * Fraction(2) ** int(e[i]))
        out.append(row)
    return out


def test_split_exact_reconstruction_and_digit_bounds():
    rng = np.random.default_rng(5)
    # rows spread over many binades, including zeros, powers of two and subnormals
    X = rng.uniform(-1, 1, (6, 9)) * np.exp2(rng.integers(-40, 40, (6, 9)))
    X[1, :] = 0.0
    X[2, 3] = 2.0 ** -1074
    X[2, 4] = -3 * 2.0 ** -1070
    X[3, :] = 2.0 ** 300
    X[4, 0] = -0.0
    # within a row the spread is < 2^80, so 53 + 80 bits -> 19 digits of 7 bits are exact
    X[2, :] = np.where(np.abs(X[2, :]) > 0, X[2, :], 1e-300)
    X[2, :] = X[2, :] * 0 + np.array([1e-300, 3e-301, -7e-302, 2.0 ** -1000, 5e-299, 1e-300, 2e-300, 3e-300, 4e-300])
    s = 20
    e, D = oracle.split(X, s)
    assert D.dtype == np.int8 and np.abs(D.astype(int)).max() <= 127
    R = reconstruct(e, D)
    for i in range(X.shape[0]):
        for l in range(X.shape[1]):
            assert R[i][l] == Fraction(float(X[i, l])), (i, l)
    assert e[1] == 0 and not D[:, 1, :].any()          # zero row
    assert (D[:, 3, :] == np.array([64] + [0] * (s - 1))[:, None]).all()  # 2^300 -> digit 64, rest 0
    assert e[3] == 301


def test_split_sign_coherence_prefix_and_residual():
    rng = np.random.default_rng(6)
    X = rng.normal(size=(8, 33)) * np.exp(3 * rng.normal(size=(8, 33)))
    e8, D8 = oracle.split(X, 8)
    e3, D3 = oracle.split(X, 3)
    assert (e8 == e3).all() and (D8[:3] == D3).all()   # prefix property
    sg = np.sign(X)[None, :, :]
    assert ((D8 == 0) | (np.sign(D8) == sg)).all()   # digits carry the sign of the entry
    R3 = reconstruct(e3, D3)
    for i in range(8):
        # |a'| in [1/2, 1) for the row max, |a' - sum| < 2^-21, truncation toward zero
        assert max(abs(Fraction(float(x))) for x in X[i]) / Fraction(2) ** int(e3[i]) >= Fraction(1, 2)
        for l in range(33):
            a = Fraction(float(X[i, l]))
            r = a - R3[i][l]
            assert abs(r) < Fraction(2) ** (int(e3[i]) - 21)
            assert r == 0 or (r > 0) == (a > 0)


def test_split_closed_form_values():
    # a' = 1 - 2^-14 has base-128 digits 127, 127, then zeros; 0.75 -> 96 (0.75*128), -0.5 -> -64
    X = np.array([[1.0 - 2.0 ** -14, 0.75, -0.5, 2.0 ** -7]])
    e, D = oracle.split(X, 3)
    assert e[0] == 0
    assert D[:, 0, 0].tolist() == [127, 127, 0]
    assert D[:, 0, 1].tolist() == [96, 0, 0]
    assert D[:, 0, 2].tolist() == [-64, 0, 0]
    assert D[:, 0, 3].tolist() == [1, 0, 0]


def test_split_transposed_and_columns():
    rng = np.random.default_rng(7)
    X = rng.normal(size=(5, 4))
    e1, D1 = oracle.split(X, 4, "N")
    e2, D2 = oracle.split(np.asfortranarray(X.T), 4, "T")
    assert (e1 == e2).all() and (D1 == D2).all()
    f, DB = oracle.split_cols(X, 4)          # columns of X
    e3, D3 = oracle.split(np.asfortranarray(X.T), 4, "N")
    assert (f == e3).all() and (DB == D3).all()


def test_zsplit_shared_exponent_and_conjugation():
    rng = np.random.default_rng(8)
    X = rng.normal(size=(3, 5)) + 1j * rng.normal(size=(3, 5)) * 8
    e, D = oracle.zsplit(X, 9, "N")
    for i in range(3):
        mx = max(max(abs(z.real), abs(z.imag)) for z in X[i])
        assert e[i] == math.frexp(mx)[1]
    R = reconstruct(np.repeat(e, 2), D)
    for i in range(3):
        for l in range(5):
            # 9 digits = 63 bits cover 53 bits + the Re/Im exponent gap only approximately:
            assert abs(R[2 * i][l] - Fraction(X[i, l].real)) < Fraction(2) ** (int(e[i]) - 63)
            assert abs(R[2 * i + 1][l] - Fraction(X[i, l].imag)) < Fraction(2) ** (int(e[i]) - 63)
    eC, DC = oracle.zsplit(np.asfortranarray(X.T), 9, "C")   # rows of (X^T)^H = conj(X)
    assert (eC == e).all()
    assert (DC[:, 0::2] == D[:, 0::2]).all() and (DC[:, 1::2] == -D[:, 1::2]).all()


# --------------------------------------------------------------------------- slice products
@pytest.mark.parametrize("square", [False, True])
def test_group_products_brute_force(square):
    rng = np.random.default_rng(9)
    s, m, n, k = 4, 3, 5, 7
    DA = rng.integers(-127, 128, (s, m, k)).astype(np.int8)
    DB = rng.integers(-127, 128, (s, n, k)).astype(np.int8)
    G = oracle.group_products(DA, DB, square)
    for i in range(m):
        for j in range(n):
            exp = {}
            for p in range(1, s + 1):
                for q in range(1, s + 1):
                    if not square and p + q > s + 1:
                        continue
                    acc = 0
                    for l in range(k):
                        acc += int(DA[p - 1, i, l]) * int(DB[q - 1, j, l])
                    exp[p + q] = exp.get(p + q, 0) + acc
            for g, v in exp.items():
                assert G[g - 2, i, j] == v
    assert G.shape[0] == (2 * s - 1 if square else s)


def test_group_products_extremes_no_overflow():
    s, k = 3, 4096
    DA = np.full((s, 1, k), 127, np.int8)
    DB = np.full((s, 1, k), -127, np.int8)
    G = oracle.group_products(DA, DB)
    assert G[0, 0, 0] == -127 * 127 * k and G[2, 0, 0] == -3 * 127 * 127 * k


# --------------------------------------------------------------------------- emulated GEMM
def test_emu_integer_inputs_single_slice_is_exact_matmul():
    rng = np.random.default_rng(10)
    A = rng.integers(-127, 128, (6, 11)).astype(float)
    B = rng.integers(-127, 128, (11, 4)).astype(float)
    A[:, 0] = 127.0  # row max 127 -> e = 7, a' = a/128, one 7-bit digit is exact
    B[0, :] = -127.0
    C = oracle.dgemm_emu(A, B, 1)
    assert (C == A @ B).all()


@pytest.mark.parametrize("seed", [0, 1])
def test_emu_exactly_representable_square_set_is_correctly_rounded(seed):
    # entries with <= 21 significant bits inside a 2^8 window of the row max are exact in
    # s = 5 digits; with all s^2 pairs T equals the exact product, so C = RN(AB)
    rng = np.random.default_rng(seed)
    m, k, n = 4, 6, 5
    A = rng.integers(-2 ** 20, 2 ** 20, (m, k)) * np.exp2(rng.integers(-8, 0, (m, k))) * 2.0 ** -20
    B = rng.integers(-2 ** 20, 2 ** 20, (k, n)) * np.exp2(rng.integers(-8, 0, (k, n))) * 2.0 ** -20
    C = oracle.dgemm_emu(A, B, 5, square=True)
    ex = frac_matmul(A, B)
    for i in range(m):
        for j in range(n):
            assert C[i, j] == float(ex[i][j])


def test_emu_rounding_ties_and_subnormals():
    # (1 + 2^-52)^2 = 1 + 2^-51 + 2^-104 -> RN gives 1 + 2^-51
    a = 1.0 + 2.0 ** -52
    C = oracle.dgemm_emu(np.array([[a]]), np.array([[a]]), 9, square=True)
    assert C[0, 0] == 1.0 + 2.0 ** -51
    # 1.5 * 2^-1075 is above half of the smallest subnormal -> rounds to 2^-1074
    C = oracle.dgemm_emu(np.array([[1.5 * 2.0 ** -537]]), np.array([[2.0 ** -538]]), 2, square=True)
    assert C[0, 0] == 2.0 ** -1074
    # exactly half of the smallest subnormal ties to even -> 0
    C = oracle.dgemm_emu(np.array([[2.0 ** -537]]), np.array([[2.0 ** -538]]), 2, square=True)
    assert C[0, 0] == 0.0
    # 3 * 2^-1075 (tie between 1 and 2 ulps of 2^-1074) -> even = 2 * 2^-1074
    C = oracle.dgemm_emu(np.array([[1.5 * 2.0 ** -537]]), np.array([[2.0 ** -537]]), 2, square=True)
    assert C[0, 0] == 2.0 ** -1073
    # overflow -> inf
    C = oracle.dgemm_emu(np.array([[2.0 ** 600]]), np.array([[2.0 ** 600]]), 2)
    assert C[0, 0] == np.inf


def test_znaive_small_integers_exact_with_complex_alpha_beta():
    """The plain complex GEMM on small Gaussian integers with complex alpha and beta: every
    operation is exact in FP64, so the result equals the exact complex arithmetic."""
    rng = np.random.default_rng(41)
    A = rng.integers(-4, 5, (3, 5)) + 1j * rng.integers(-4, 5, (3, 5))
    B = rng.integers(-4, 5, (5, 2)) + 1j * rng.integers(-4, 5, (5, 2))
    C0 = rng.integers(-4, 5, (3, 2)) + 1j * rng.integers(-4, 5, (3, 2))
    al, be = 2 - 3j, 0.5 + 1j
    C = oracle.zgemm_naive(A, B, alpha=al, beta=be, C=C0)
    want = [[al * sum(complex(A[i, l]) * complex(B[l, j]) for l in range(5)) + be * complex(C0[i, j])
             for j in range(2)] for i in range(3)]
    assert (C == np.array(want)).all()


def test_emu_single_rounding_at_the_subnormal_and_overflow_edges():
    """One rounding of the exact sum, also where a 53-bit rounding followed by a second one onto
    the subnormal grid (or past the largest finite value) would differ (s = 18 keeps every term).
    2^-1075 + 2^-1130 lies above half of the smallest subnormal, so RN gives 2^-1074, while
    rounding to 53 bits first gives exactly 2^-1075, whose tie goes to 0.  The largest finite
    double plus half its ulp (2^970) ties to even, which is upwards here: +inf."""
    A = np.array([[2.0 ** -500, 2.0 ** -555]])
    B = np.array([[2.0 ** -575], [2.0 ** -575]])
    assert oracle.dgemm_emu(A, B, 18)[0, 0] == 2.0 ** -1074
    assert oracle.dgemm_emu(-A, B, 18)[0, 0] == -(2.0 ** -1074)
    big = float(np.finfo(np.float64).max)
    assert big == 2.0 ** 1023 + (2.0 ** 1023 - 2.0 ** 971)
    A = np.array([[2.0 ** 1023, 2.0 ** 1023 - 2.0 ** 971, 2.0 ** 970]])
    B = np.ones((3, 1))
    assert oracle.dgemm_emu(A, B, 18)[0, 0] == np.inf
    assert oracle.dgemm_emu(A[:, :2], B[:2], 18)[0, 0] == big        # exactly the largest finite


def test_emu_triangle_matches_definition_on_tiny():
    # brute-force T from the (already pinned) digits with Python integers, then RN
    rng = np.random.default_rng(11)
    m, k, n, s = 3, 5, 4, 4
    A = rng.normal(size=(m, k)) * np.exp(2 * rng.normal(size=(m, k)))
    B = rng.normal(size=(k, n)) * np.exp(2 * rng.normal(size=(k, n)))
    e, DA = oracle.split(A, s)
    f, DB = oracle.split_cols(B, s)
    C = oracle.dgemm_emu(A, B, s)
    for i in range(m):
        for j in range(n):
            T = Fraction(0)
            for p in range(1, s + 1):
                for q in range(1, s + 2 - p):
                    d = sum(int(DA[p - 1, i, l]) * int(DB[q - 1, j, l]) for l in range(k))
                    T += Fraction(d) * Fraction(2) ** (int(e[i]) + int(f[j]) - 7 * (p + q))
            assert C[i, j] == float(T)


@pytest.mark.parametrize("s", [2, 3, 4, 5, 6, 7, 8])
def test_emu_error_within_a_priori_bound(s):
    rng = np.random.default_rng(100 + s)
    m, k, n = 24, 70, 20
    phi = 3.0
    A = (rng.uniform(size=(m, k)) - 0.5) * np.exp(phi * rng.normal(size=(m, k)))
    B = (rng.uniform(size=(k, n)) - 0.5) * np.exp(phi * rng.normal(size=(k, n)))
    C = oracle.dgemm_emu(A, B, s)
    hi, lo = oracle.dgemm_dd(A, B)
    bound = oracle.emu_bound(A, B, s) + U * np.abs(C) + 4 * k * U * U * (np.abs(A) @ np.abs(B))
    assert (np.abs((C - hi) - lo) <= bound).all()
    # triangle vs square set: the dropped pairs are also inside the bound
    Cs = oracle.dgemm_emu(A, B, s, square=True)
    assert (np.abs((Cs - hi) - lo) <= bound).all()


def test_emu_error_bound_adversarial_all_max_digits():
    # a' = 1 - 2^-7s has every digit equal to 127: the residual and the dropped pairs are maximal
    s, k = 4, 64
    rng = np.random.default_rng(12)
    val = 1.0 - 2.0 ** (-7 * s - 2)  # digits 127 x s and a positive residual
    A = val * rng.choice([-1.0, 1.0], size=(8, k))
    B = val * rng.choice([-1.0, 1.0], size=(k, 8))
    C = oracle.dgemm_emu(A, B, s)
    hi, lo = oracle.dgemm_dd(A, B)
    bound = oracle.emu_bound(A, B, s) + U * np.abs(C)
    err = np.abs((C - hi) - lo)
    assert (err <= bound).all() and err.max() > 0


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_emu_transposes_alpha_beta(ta, tb):
    rng = np.random.default_rng(13)
    m, k, n, s = 9, 13, 7, 6
    A = rng.normal(size=(m, k) if ta == "N" else (k, m))
    B = rng.normal(size=(k, n) if tb == "N" else (n, k))
    opA = A if ta == "N" else A.T
    opB = B if tb == "N" else B.T
    C0 = rng.normal(size=(m, n))
    t = oracle.dgemm_emu(np.asfortranarray(opA), np.asfortranarray(opB), s)
    C = oracle.dgemm_emu(A, B, s, ta, tb, alpha=-0.75, beta=0.5, C=C0)
    exp = np.array([[fma_exact(-0.75, t[i, j], 0.5 * C0[i, j]) for j in range(n)] for i in range(m)])
    assert (C == exp).all()
    np.testing.assert_allclose(C, -0.75 * opA @ opB + 0.5 * C0, rtol=0, atol=1e-9)


def fma_exact(x, y, z):
    """RN(x y + z) with one rounding: the sum formed exactly in rationals, then rounded to the
    nearest double (CPython's int / int division rounds correctly)."""
    return float(Fraction(x) * Fraction(y) + Fraction(z))


def test_emu_alpha_beta_single_rounding_directed():
    """C = RN(alpha t + RN(beta C_old)) in one rounding (the fma reading of the update): with
    alpha = t = 1 + 2^-30 and beta C_old = -(1 + 2^-29), the exact update is 2^-60, while
    rounding alpha t first would give 0."""
    x = 1.0 + 2.0 ** -30
    A, B = np.array([[x]]), np.array([[1.0]])
    C0 = np.array([[1.0 + 2.0 ** -29]])
    C = oracle.dgemm_emu(A, B, 6, alpha=x, beta=-1.0, C=C0)   # 31 significant bits: exact at s = 6
    assert C[0, 0] == 2.0 ** -60 == fma_exact(x, x, -(1.0 + 2.0 ** -29))


def test_emu_trend_error_falls_per_slice():
    # qualitative trend of Table 1: each added slice cuts the error by tens to hundreds of
    # times (parity unpinned for the application numbers themselves)
    rng = np.random.default_rng(14)
    A = rng.uniform(-1, 1, (32, 64))
    B = rng.uniform(-1, 1, (64, 32))
    errs = [oracle.rel_err_vs_dd(oracle.dgemm_emu(A, B, s), A, B) for s in range(2, 8)]
    for a, b in zip(errs, errs[1:]):
        assert b < a / 30


# --------------------------------------------------------------------------- complex
def frac_cmatmul(A, B):
    m, k = A.shape
    n = B.shape[1]
    re = [[sum(Fraction(A[i, l].real) * Fraction(B[l, j].real) - Fraction(A[i, l].imag) * Fraction(B[l, j].imag)
               for l in range(k)) for j in range(n)] for i in range(m)]
    im = [[sum(Fraction(A[i, l].real) * Fraction(B[l, j].imag) + Fraction(A[i, l].imag) * Fraction(B[l, j].real)
               for l in range(k)) for j in range(n)] for i in range(m)]
    return re, im


def test_zdd_matches_exact_rationals():
    rng = np.random.default_rng(15)
    A = rng.normal(size=(3, 6)) + 1j * rng.normal(size=(3, 6))
    B = rng.normal(size=(6, 2)) + 1j * rng.normal(size=(6, 2))
    rh, rl, ih, il = oracle.zgemm_dd(A, B)
    re, im = frac_cmatmul(A, B)
    for i in range(3):
        for j in range(2):
            assert abs(Fraction(rh[i, j]) + Fraction(rl[i, j]) - re[i][j]) < Fraction(2) ** -95
            assert abs(Fraction(ih[i, j]) + Fraction(il[i, j]) - im[i][j]) < Fraction(2) ** -95


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("C", "N"), ("N", "T"), ("N", "C"), ("C", "C")])
def test_zemu_exact_inputs_correctly_rounded(ta, tb):
    # parts with <= 14 significant bits inside a 2^6 window of the complex row max are exact
    # in 3 digits... use s = 4 and the 4 real sub-products: T is exact, so C = RN(AB) per part
    rng = np.random.default_rng(16)
    m, k, n = 3, 5, 4

    def mk(shape):
        re = rng.integers(-2 ** 13, 2 ** 13, shape) * np.exp2(rng.integers(-6, 0, shape)) * 2.0 ** -13
        im = rng.integers(-2 ** 13, 2 ** 13, shape) * np.exp2(rng.integers(-6, 0, shape)) * 2.0 ** -13
        return re + 1j * im

    opA, opB = mk((m, k)), mk((k, n))
    A = opA if ta == "N" else (opA.T if ta == "T" else opA.conj().T)
    B = opB if tb == "N" else (opB.T if tb == "T" else opB.conj().T)
    # the triangle set with s digits covers every pair p+q <= s+1; digits here need <= 3 planes,
    # so s = 5 keeps all nonzero pairs (p, q <= 3 -> p + q <= 6 = s + 1)
    C = oracle.zgemm_emu(A, B, 5, ta, tb)
    re, im = frac_cmatmul(opA, opB)
    for i in range(m):
        for j in range(n):
            assert C[i, j].real == float(re[i][j]) and C[i, j].imag == float(im[i][j])


def test_zemu_error_bound_and_alpha_beta():
    rng = np.random.default_rng(17)
    m, k, n, s = 8, 20, 6, 7
    A = rng.normal(size=(m, k)) + 1j * rng.normal(size=(m, k))
    B = rng.normal(size=(k, n)) + 1j * rng.normal(size=(k, n))
    C = oracle.zgemm_emu(A, B, s)
    rh, rl, ih, il = oracle.zgemm_dd(A, B)
    scale = np.abs(A.real) @ np.abs(B.real) + np.abs(A.imag) @ np.abs(B.imag) + \
        np.abs(A.real) @ np.abs(B.imag) + np.abs(A.imag) @ np.abs(B.real)
    err = np.maximum(np.abs(C.real - rh - rl), np.abs(C.imag - ih - il)) / scale
    assert err.max() < 4 * (s + 2) * 2.0 ** (-7 * s) * 4
    al, be = 0.5 - 2j, 1.5 + 0.25j
    C0 = rng.normal(size=(m, n)) + 1j * rng.normal(size=(m, n))
    C2 = oracle.zgemm_emu(A, B, s, alpha=al, beta=be, C=C0)
    np.testing.assert_allclose(C2, al * C + be * C0, rtol=1e-13, atol=1e-13)


def test_zemu_alpha_beta_single_rounding_directed():
    """Complex update in the fma order: Re = RN(alpha_r t_r - RN(alpha_i t_i)) and
    Im = RN(alpha_r t_i + RN(alpha_i t_r)).  With t = (1 + 2^-30) + i (1 + 2^-29) and alpha =
    (1 + 2^-30) + i, the exact real part is 2^-60, which rounding alpha_r t_r first would lose."""
    x, y = 1.0 + 2.0 ** -30, 1.0 + 2.0 ** -29
    A, B = np.array([[complex(x, y)]]), np.array([[1.0 + 0j]])
    C = oracle.zgemm_emu(A, B, 6, alpha=complex(x, 1.0))   # 31 significant bits: exact at s = 6
    assert C[0, 0].real == 2.0 ** -60 == fma_exact(x, x, -(1.0 * y))
    assert C[0, 0].imag == fma_exact(x, y, 1.0 * x)
    be = complex(1.0, -(1.0 + 2.0 ** -30))
    C0 = np.array([[complex(x, 2.0)]])
    C = oracle.zgemm_emu(A, B, 6, alpha=complex(x, 1.0), beta=be, C=C0)
    br = fma_exact(be.real, C0[0, 0].real, -(be.imag * C0[0, 0].imag))
    bi = fma_exact(be.real, C0[0, 0].imag, be.imag * C0[0, 0].real)
    assert C[0, 0].real == 2.0 ** -60 + br and C[0, 0].imag == fma_exact(x, y, 1.0 * x) + bi


def test_zemu_beta_single_rounding_directed():
    """beta C_old in the fma order as well: Re = RN(beta_r c_r - RN(beta_i c_i)).  With
    beta = (1 + 2^-30) + i, C_old = (1 + 2^-30) + i (1 + 2^-29) and a zero product, the exact
    real part is 2^-60, which rounding beta_r c_r first would lose."""
    x, y = 1.0 + 2.0 ** -30, 1.0 + 2.0 ** -29
    C0 = np.array([[complex(x, y)]])
    C = oracle.zgemm_emu(np.array([[0j]]), np.array([[1.0 + 0j]]), 4, beta=complex(x, 1.0), C=C0)
    assert C[0, 0].real == 2.0 ** -60 == fma_exact(x, x, -(1.0 * y))
    assert C[0, 0].imag == fma_exact(x, y, 1.0 * x)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("C", "N"), ("N", "T"), ("N", "C"), ("C", "T")])
def test_z3m_small_integers_exact_with_alpha_beta(ta, tb):
    """3M on small integers: every emulated product, difference and alpha/beta step is exact, so
    the result is the exact complex product (Python integers) -- a wrong sign or operand in the
    combine, a missing conjugation or a transposed operand changes it."""
    rng = np.random.default_rng(31)
    m, k, n = 4, 6, 5
    opA = rng.integers(-64, 65, (m, k)) + 1j * rng.integers(-64, 65, (m, k))
    opB = rng.integers(-64, 65, (k, n)) + 1j * rng.integers(-64, 65, (k, n))
    A = opA if ta == "N" else (opA.T if ta == "T" else opA.conj().T)
    B = opB if tb == "N" else (opB.T if tb == "T" else opB.conj().T)
    C0 = rng.integers(-8, 9, (m, n)) + 1j * rng.integers(-8, 9, (m, n))
    al, be = 2 - 1j, 0.5 + 0.25j
    C = oracle.zgemm3m_emu(np.asfortranarray(A), np.asfortranarray(B), 4, ta, tb, al, be, C0)
    for i in range(m):
        for j in range(n):
            re = sum(int(opA[i, l].real) * int(opB[l, j].real) - int(opA[i, l].imag) * int(opB[l, j].imag)
                     for l in range(k))
            im = sum(int(opA[i, l].real) * int(opB[l, j].imag) + int(opA[i, l].imag) * int(opB[l, j].real)
                     for l in range(k))
            er = Fraction(2) * re + im + Fraction(1, 2) * int(C0[i, j].real) - Fraction(1, 4) * int(C0[i, j].imag)
            ei = Fraction(2) * im - re + Fraction(1, 2) * int(C0[i, j].imag) + Fraction(1, 4) * int(C0[i, j].real)
            assert Fraction(C[i, j].real) == er and Fraction(C[i, j].imag) == ei, (i, j)


@pytest.mark.parametrize("s", [3, 5, 7, 9])
def test_z3m_error_within_its_bound(s):
    """The 3M result stays within its a priori bound (emulation error of the three real products,
    the rounding of Ar + Ai and Br + Bi, and the roundings of the combine), per part, against the
    double-double product, on inputs with wide exponent spreads and cancellation in the
    imaginary part."""
    rng = np.random.default_rng(32 + s)
    m, k, n = 9, 40, 7
    A = (rng.uniform(-1, 1, (m, k)) + 1j * rng.uniform(-1, 1, (m, k))) * np.exp(rng.normal(0, 2, (m, k)))
    B = (rng.uniform(-1, 1, (k, n)) + 1j * rng.uniform(-1, 1, (k, n))) * np.exp(rng.normal(0, 2, (k, n)))
    A[:, :3] = A[:, :3].real - 1j * A[:, :3].real  # Re + Im = 0 on some entries: Sa has zeros
    C = oracle.zgemm3m_emu(A, B, s)
    rh, rl, ih, il = oracle.zgemm_dd(A, B)
    bre, bim = oracle.zgemm3m_bound(A, B, s)
    assert (np.abs(C.real - rh - rl) <= bre).all()
    assert (np.abs(C.imag - ih - il) <= bim).all()
    # the bound is not vacuous: at these s it sits far below the products' magnitude
    assert (bim < 1e-1 * oracle.abs_product(np.abs(A.real) + np.abs(A.imag), np.abs(B.real) + np.abs(B.imag))).all()


def test_z3m_bound_covers_an_error_of_the_sum_product_alone():
    """A directed 3M case whose imaginary error comes from the third product only: Ar = Bi = 1,
    Ai = Br = 2^-30 are exact in one digit each (P1 = P2 = 2^-30 exactly), while
    Sa = Sb = 1 + 2^-30 lose their 2^-30 parts at s = 3, so P3 = 1 and Im = RN(RN(1 - 2^-30)
    - 2^-30) = 1 - 2^-29 against the exact 1 + 2^-60.  The bound must cover that error, which
    the other terms of the bound (each near 2^-46 here) cannot."""
    t = 2.0 ** -30
    A, B = np.array([[complex(1.0, t)]]), np.array([[complex(t, 1.0)]])
    C = oracle.zgemm3m_emu(A, B, 3)
    assert C[0, 0].imag == 1.0 - 2.0 * t and C[0, 0].real == 0.0
    err = abs(Fraction(C[0, 0].imag) - (1 + Fraction(t) ** 2))
    bre, bim = oracle.zgemm3m_bound(A, B, 3)
    assert Fraction(float(bim[0, 0])) >= err > Fraction(t)
    assert bre[0, 0] >= abs(Fraction(C[0, 0].real) - (Fraction(t) - Fraction(t)))


def test_rel_err_metric_closed_form():
    """max |C - C_dd| / (|alpha| |A||B| + |beta| |C0|): with A = B = 1, alpha = 4, beta = -2,
    C0 = 3, the exact update is 4 - 6 = -2, so C = -2 + 2^-40 has error 2^-40 over the scale
    4 + 6 = 10; a zero-scale entry with a zero difference counts 0."""
    A, B = np.array([[1.0, 0.0]]), np.array([[1.0, 0.0], [0.0, 0.0]])
    C0 = np.array([[3.0, 0.0]])
    C = np.array([[-2.0 + 2.0 ** -40, 0.0]])
    r = oracle.rel_err_vs_dd(C, A, B, alpha=4.0, beta=-2.0, C0=C0)
    assert r == 2.0 ** -40 / 10
    assert oracle.rel_err_vs_dd(np.array([[2.0 ** -40 + 1.0, 0.0]]), A, B) == 2.0 ** -40


def test_kkr_kappa_variant_has_the_requested_condition_number():
    """The KKR-like stand-in's conditioned variant: the cached diagonal shift puts cond_2(A)
    within a factor 1.5 of 1e8 (SVD on the host), and B is the unshifted-workload's B."""
    from paper_2503_22875_gb300 import workloads
    A, B = workloads.kkr_kappa_pair(113, 32, seed=3, kappa=1e8)
    A0, B0 = workloads.kkr_like_pair(113, 32, seed=3)
    assert np.array_equal(B, B0)
    off = ~np.eye(A.shape[0], dtype=bool)
    assert np.array_equal(A[off], A0[off])  # only the diagonal shift differs
    sv = np.linalg.svd(A, compute_uv=False)
    assert 1e8 / 1.5 <= sv[0] / sv[-1] <= 1e8 * 1.5


# ------------------------------------------------------------------ worked example (golden)
GOLDEN = __import__("pathlib").Path(__file__).parent / "golden"


def read_golden(name):
    """key -> list of rows of Fractions from a tests/golden fixture ('a b ; c d' = two rows)."""
    out = {}
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, vals = line.split(":", 1)
        out[key.strip()] = [[Fraction(v) for v in row.split()] for row in vals.split(";")]
    return out


def test_worked_example_split_groups_and_triangle_by_hand():
    """The hand-derived example of tests/golden/worked_example_split_triangle.txt (Sec. 2.2):
    exponents, digits and group products equal the derivation; s = 2 drops exactly the pair
    (2, 2) of group 4 (+15 / 2^28 on entry (1, 1)), and s = 3 gives the exact product."""
    g = read_golden("worked_example_split_triangle.txt")
    A = np.array([[float(x) for x in r] for r in g["A"]])
    B = np.array([[float(x) for x in r] for r in g["B"]])
    e, DA = oracle.split(A, 3)
    f, DB = oracle.split_cols(B, 3)
    assert e.tolist() == [int(x) for x in g["e"][0]]
    assert f.tolist() == [int(x) for x in g["f"][0]]
    for t in range(3):
        assert DA[t].tolist() == [[int(x) for x in r] for r in g[f"DA_{t + 1}"]]
        assert DB[t].tolist() == [[int(x) for x in r] for r in g[f"DB_{t + 1}"]]
    G = oracle.group_products(DA, DB)
    for gi in range(3):
        assert G[gi].tolist() == [[int(x) for x in r] for r in g[f"G_s3_g{gi + 2}"]]
    exact = frac_matmul(A, B)
    assert exact == g["C_exact"]
    for s in (2, 3):
        C = oracle.dgemm_emu(A, B, s)
        assert [[Fraction(float(x)) for x in r] for r in C] == g[f"C_s{s}"]
    # the dropped pair, by itself: s = 2 minus the exact product on entry (1, 1)
    assert Fraction(float(oracle.dgemm_emu(A, B, 2)[0, 0])) - exact[0][0] == Fraction(15, 2 ** 28)


@pytest.mark.parametrize("ta", ["N", "C"])
def test_worked_example_complex_by_hand(ta):
    """The one-element complex example of the same fixture: shared exponent, conjugation of the
    imaginary digits for op = 'C', and the exact product at s = 1."""
    g = read_golden("worked_example_split_triangle.txt")
    a = complex(float(g["zA"][0][0]), float(g["zA"][0][1]))
    b = complex(float(g["zB"][0][0]), float(g["zB"][0][1]))
    C = oracle.zgemm_emu(np.array([[a]]), np.array([[b]]), 1, transa=ta)
    want = g[f"zC_{ta}"][0]
    assert (Fraction(C[0, 0].real), Fraction(C[0, 0].imag)) == (want[0], want[1])
