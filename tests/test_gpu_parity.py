"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same seeded inputs.

  * split exponents and INT8 digits: bit-exact (integer work)
  * integer group products G_g from the tensor-core kernel: bit-exact
  * emulated DGEMM / ZGEMM: bit-exact where the epilogue's exact int64 windows cover every group
    (at most two windows: s <= 10 at any k, s <= 12 for k <= 512), else within a tolerance
    derived from the FP64 continuation (one rounding per later window) -- |C_gpu - C_oracle| <=
    4 (s + 2) u |alpha| (|A||B|) + 2 u |C| + u |beta| |C0| -- and within the a priori bound of
    the method against double-double.
  * native FP64 kernel: within gamma_k of double-double.
"""
import numpy as np
import pytest

import oracle
from paper_2503_22875_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module")
def ozg():
    from paper_2503_22875_gb300 import build, ozg
    build.build()
    ozg.load()
    return ozg


@pytest.fixture(scope="module")
def ctx(ozg):
    c = ozg.Context()
    yield c
    c.close()


def dev(ozg, x):
    return ozg.to_device(x)


def host(ozg, t, m, n):
    return ozg.from_device(t, m, n)


def wide(shape, phi, seed, zeros=True):
    g = workloads.rng(seed)
    X = workloads.wide_exponent(shape, phi, g)
    if zeros and X.size > 3:
        X.flat[:: max(7, X.size // 5)] = 0.0
    return np.asfortranarray(X)


# ----------------------------------------------------------------------------- split
@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("rows,k,s", [(1, 1, 1), (37, 70, 7), (200, 131, 3), (64, 1000, 12), (5, 9, 18)])
def test_split_bit_exact(ozg, ctx, trans, rows, k, s):
    X = wide((rows, k) if trans == "N" else (k, rows), 6.0, rows * 1000 + k)
    if X.size > 10:
        X.flat[3] = 2.0 ** -1074
        X.flat[5] = -3.5e-310
    dX = dev(ozg, X)
    e = torch.empty(rows, dtype=torch.int32, device="cuda")
    d = torch.empty((s, rows, k), dtype=torch.int8, device="cuda")
    ctx.debug_split(trans, rows, k, dX, X.shape[0], s, e, d)
    e_o, d_o = oracle.split(X, s, trans)
    assert np.array_equal(e.cpu().numpy(), e_o)
    assert np.array_equal(d.cpu().numpy(), d_o)


@pytest.mark.parametrize("trans", ["N", "T", "C"])
def test_zsplit_bit_exact(ozg, ctx, trans):
    rows, k, s = 45, 77, 9
    shape = (rows, k) if trans == "N" else (k, rows)
    X = wide(shape, 3.0, 5) + 1j * wide(shape, 3.0, 6)
    dX = dev(ozg, X)
    e = torch.empty(rows, dtype=torch.int32, device="cuda")
    d = torch.empty((s, 2 * rows, k), dtype=torch.int8, device="cuda")
    ctx.debug_split(trans, rows, k, dX, X.shape[0], s, e, d, complex_=True)
    e_o, d_o = oracle.zsplit(X, s, trans)
    assert np.array_equal(e.cpu().numpy(), e_o)
    assert np.array_equal(d.cpu().numpy(), d_o)


# ----------------------------------------------------------------------------- group products
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("m,n,k,s", [(128, 256, 64, 3), (130, 300, 1100, 4), (7, 5, 3, 7), (257, 513, 200, 8)])
def test_group_products_bit_exact(ozg, ctx, ta, tb, m, n, k, s):
    A = wide((m, k) if ta == "N" else (k, m), 2.0, m + 1)
    B = wide((k, n) if tb == "N" else (n, k), 2.0, n + 2)
    G = torch.empty((s, m, n), dtype=torch.int64, device="cuda")
    ctx.debug_group_products(ta, tb, m, n, k, dev(ozg, A), A.shape[0], dev(ozg, B), B.shape[0], s, G)
    _, DA = oracle.split(A, s, ta)
    _, DB = oracle.split(B, s, "T" if tb == "N" else "N")
    G_o = oracle.group_products(DA, DB)
    assert np.array_equal(G.cpu().numpy(), G_o)


def test_group_products_max_digits_chain_boundary(ozg, ctx):
    # every digit +-127 and k crossing several 1024-product chains: the largest exact FP32 sums
    s, k = 4, 1000
    v = 1.0 - 2.0 ** (-7 * s - 3)
    g = workloads.rng(9)
    A = np.asfortranarray(v * g.choice([-1.0, 1.0], size=(130, k)))
    A[:, :] = np.abs(A)  # all positive: chains reach the largest magnitude
    B = np.asfortranarray(np.full((k, 260), v))
    G = torch.empty((s, 130, 260), dtype=torch.int64, device="cuda")
    ctx.debug_group_products("N", "N", 130, 260, k, dev(ozg, A), 130, dev(ozg, B), k, s, G)
    _, DA = oracle.split(A, s)
    _, DB = oracle.split_cols(B, s)
    G_o = oracle.group_products(DA, DB)
    assert G_o[s - 1].max() == s * k * 127 * 127
    assert np.array_equal(G.cpu().numpy(), G_o)


# The epilogue keeps each group's running sum in int32 and folds it into the int64 window
# every 64 accumulation chains of 1024 products (65,536 products, real) or every 32 chains
# (complex, where Re = P_rr - P_ii doubles the magnitude).  With every digit 127 and one sign,
# the last group of s = 4 at these k holds more than 2^31 - 1 in total, so a missing or late fold
# overflows.  v = 1 - 2^-28 has the digits 127, 127, 127, 127 at s = 4.
FOLD_S = 4
FOLD_V = 1.0 - 2.0 ** -28


def fold_operands(m, n, k, mixed_rows=8, seed=7):
    """All-127 digits of one sign, except `mixed_rows` rows of A that mix signs and spreads (so
    that a fold is also checked on ordinary data)."""
    A = np.full((m, k), FOLD_V)
    A[:mixed_rows] = wide((mixed_rows, k), 2.0, seed, zeros=False)
    B = np.full((k, n), FOLD_V)
    return np.asfortranarray(A), np.asfortranarray(B)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N")])
def test_group_products_cross_int32_fold(ozg, ctx, ta, tb):
    m, n, k, s = 40, 33, 34000, FOLD_S
    A, B = fold_operands(m, n, k)
    A = np.asfortranarray(A.T) if ta == "T" else A
    G = torch.empty((s, m, n), dtype=torch.int64, device="cuda")
    ctx.debug_group_products(ta, tb, m, n, k, dev(ozg, A), A.shape[0], dev(ozg, B), k, s, G)
    _, DA = oracle.split(A, s, ta)
    _, DB = oracle.split_cols(B, s)
    G_o = oracle.group_products(DA, DB)
    assert G_o[s - 1].max() == s * k * 127 * 127 > 2 ** 31 - 1  # the last group needs the fold
    assert s * k > 64 * 1024                                     # it spans more than 64 chains
    assert np.array_equal(G.cpu().numpy(), G_o)


def test_dgemm_cross_int32_fold_bit_exact(ozg, ctx):
    """The same operands through the emulated DGEMM (one int64 window, so the oracle's definition
    bit for bit), single call and grouped launch, both tile widths, CTA pairs and stacked group
    pairs (whose chains go straight into int64 windows, with no int32 fold)."""
    m, n, k, s = 40, 33, 34000, FOLD_S
    A, B = fold_operands(m, n, k)
    assert windows(s, k) == 1
    E = oracle.dgemm_emu(A, B, s)
    dA, dB = dev(ozg, A), dev(ozg, B)
    for variant in (0, 1, 4, 5):
        ctx.set_tile_variant(variant)
        try:
            dC = torch.zeros((n, m), dtype=torch.float64, device="cuda")
            ctx.dgemm("N", "N", m, n, k, 1.0, dA, m, dB, k, 0.0, dC, m, s)
            ctx.sync()
            assert np.array_equal(host(ozg, dC, m, n), E), variant
            dG = torch.zeros((n, m), dtype=torch.float64, device="cuda")
            ctx.dgemm_grouped([("N", "N", m, n, k, 1.0, dA, m, dB, k, 0.0, dG, m)], [s])
            ctx.sync()
            assert np.array_equal(host(ozg, dG, m, n), E), variant
        finally:
            ctx.set_tile_variant(-1)


@pytest.mark.parametrize("ta", ["N", "C"])
def test_zgemm_cross_complex_int32_fold_bit_exact(ozg, ctx, ta):
    """Complex: Re(A) = Im(A) = v and Re(B) = -Im(B) = v make Re = P_rr - P_ii twice the largest
    real sub-product; at k = 17000 the last group of s = 4 holds 2 * 4 * k * 127^2 > 2^31 - 1, so
    the 32-chain complex fold is needed.  Some rows mix signs and spreads."""
    m, n, k, s = 24, 20, 17000, FOLD_S
    A = np.full((m, k), FOLD_V * (1 + 1j))
    A[:4] = wide((4, k), 2.0, 31, zeros=False) + 1j * wide((4, k), 2.0, 32, zeros=False)
    B = np.asfortranarray(np.full((k, n), FOLD_V * (1 - 1j)))
    assert windows(s, k, cplx=True) == 1
    assert 2 * s * k * 127 * 127 > 2 ** 31 - 1
    Aop = np.asfortranarray(A.conj().T) if ta == "C" else np.asfortranarray(A)
    dC = torch.zeros((n, m), dtype=torch.complex128, device="cuda")
    ctx.zgemm(ta, "N", m, n, k, 1.0, dev(ozg, Aop), Aop.shape[0], dev(ozg, B), k, 0.0, dC, m, s)
    ctx.sync()
    E = oracle.zgemm_emu(Aop, B, s, ta, "N")
    assert np.array_equal(host(ozg, dC, m, n), E)


# ----------------------------------------------------------------------------- emulated DGEMM
def check_dgemm(C, A, B, s, ta, tb, alpha, beta, C0):
    E = oracle.dgemm_emu(A, B, s, ta, tb, alpha, beta, C0)
    AB = oracle.abs_product(A, B, ta, tb)
    tol = 4 * (s + 2) * U * abs(alpha) * AB + 2 * U * np.abs(E)
    if C0 is not None and beta != 0:
        tol = tol + 2 * U * abs(beta) * np.abs(C0)
    diff = np.abs(C - E)
    assert (diff <= tol).all(), f"max excess {(diff - tol).max():.3e}"
    # and the method's own a priori bound against double-double
    hi, lo = oracle.dgemm_dd(A, B, ta, tb, alpha, beta, C0)
    bnd = abs(alpha) * (oracle.emu_bound(A, B, s, ta, tb) + (s + 4) * U * AB) + 2 * U * np.abs(hi)
    if C0 is not None and beta != 0:
        bnd = bnd + 2 * U * abs(beta) * np.abs(C0)
    assert (np.abs((C - hi) - lo) <= bnd).all()


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("m,n,k,s", [(256, 256, 256, 7), (300, 520, 130, 3), (33, 257, 31, 5), (129, 255, 1500, 6),
                                     (1, 1, 1, 1), (17, 600, 64, 10)])
def test_dgemm_parity(ozg, ctx, ta, tb, m, n, k, s):
    A = wide((m, k) if ta == "N" else (k, m), 2.0, 11 * m + k)
    B = wide((k, n) if tb == "N" else (n, k), 2.0, 13 * n + k)
    C = torch.zeros((n, m), dtype=torch.float64, device="cuda")
    rep = ctx.dgemm(ta, tb, m, n, k, 1.0, dev(ozg, A), A.shape[0], dev(ozg, B), B.shape[0], 0.0, C, m, s,
                    report=True)
    assert rep.slices_used == s and rep.nonfinite == 0
    ctx.sync()
    check_dgemm(host(ozg, C, m, n), A, B, s, ta, tb, 1.0, 0.0, None)


@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (-0.5, 0.25), (2.0, -1.0), (3.0, 0.0)])
def test_dgemm_alpha_beta_and_ldc(ozg, ctx, alpha, beta):
    m, n, k, s = 150, 270, 90, 7
    A, B = workloads.uniform_pair(m, n, k, seed=21)
    ldc = m + 5
    C0 = np.asfortranarray(workloads.rng(22).uniform(-1, 1, (ldc, n)))
    dC = dev(ozg, C0)
    ctx.dgemm("N", "N", m, n, k, alpha, dev(ozg, A), m, dev(ozg, B), k, beta, dC, ldc, s)
    ctx.sync()
    Cg = host(ozg, dC, ldc, n)
    check_dgemm(Cg[:m], A, B, s, "N", "N", alpha, beta, C0[:m])
    assert np.array_equal(Cg[m:], C0[m:])  # rows between m and ldc untouched


def test_dgemm_lda_padding_and_beta_zero_ignores_nan(ozg, ctx):
    m, n, k, s = 100, 90, 80, 6
    Af = wide((m + 3, k), 1.0, 31)
    Bf = wide((k + 2, n), 1.0, 32)
    C0 = np.full((m, n), np.nan, order="F")
    dC = dev(ozg, C0)
    ctx.dgemm("N", "N", m, n, k, 1.0, dev(ozg, Af), m + 3, dev(ozg, Bf), k + 2, 0.0, dC, m, s)
    ctx.sync()
    C = host(ozg, dC, m, n)
    assert np.isfinite(C).all()
    check_dgemm(C, np.asfortranarray(Af[:m]), np.asfortranarray(Bf[:k]), s, "N", "N", 1.0, 0.0, None)


def test_dgemm_quick_returns(ozg, ctx):
    m, n, k = 40, 30, 20
    A, B = workloads.uniform_pair(m, n, k, seed=41)
    C0 = np.asfortranarray(workloads.rng(42).uniform(-1, 1, (m, n)))
    for alpha, beta, kk, expect in [(0.0, 1.0, k, C0), (1.0, 1.0, 0, C0), (0.0, 2.5, k, 2.5 * C0),
                                    (1.0, 0.0, 0, np.zeros_like(C0))]:
        dC = dev(ozg, C0)
        ctx.dgemm("N", "N", m, n, kk, alpha, dev(ozg, A), m, dev(ozg, B), max(kk, 1), beta, dC, m, 7)
        ctx.sync()
        assert np.array_equal(host(ozg, dC, m, n), expect)
    dC = dev(ozg, C0)
    ctx.dgemm("N", "N", 0, n, k, 1.0, dev(ozg, A), 1, dev(ozg, B), k, 0.0, dC, 1, 7)  # m == 0: no-op
    ctx.sync()
    assert np.array_equal(host(ozg, dC, m, n), C0)


def test_nonfinite_routes_to_native(ozg, ctx):
    m, n, k = 64, 48, 40
    A, B = workloads.uniform_pair(m, n, k, seed=51)
    A[3, 7] = np.inf
    B[2, 5] = np.nan
    dC = torch.zeros((n, m), dtype=torch.float64, device="cuda")
    rep = ctx.dgemm("N", "N", m, n, k, 1.0, dev(ozg, A), m, dev(ozg, B), k, 0.0, dC, m, 7, report=True)
    assert rep.nonfinite == 1 and rep.slices_used == -1
    C = host(ozg, dC, m, n)
    ref = oracle.dgemm_naive(A, B)
    same = (np.isnan(C) == np.isnan(ref)) & (np.isinf(C) == np.isinf(ref))
    assert same.all()
    fin = np.isfinite(ref)
    np.testing.assert_allclose(C[fin], ref[fin], rtol=1e-13, atol=1e-13)


def test_slices_monotone_error(ozg, ctx):
    m = n = k = 192
    A, B = workloads.wide_exponent_pair(m, n, k, 2.0, seed=61)
    dA, dB = dev(ozg, A), dev(ozg, B)
    errs = []
    for s in range(3, 10):
        C = torch.zeros((n, m), dtype=torch.float64, device="cuda")
        ctx.dgemm("N", "N", m, n, k, 1.0, dA, m, dB, k, 0.0, C, m, s)
        ctx.sync()
        errs.append(oracle.rel_err_vs_dd(host(ozg, C, m, n), A, B))
    for a, b in zip(errs, errs[1:]):
        assert b <= a / 20 or b < 1e-15


# ----------------------------------------------------------------------------- emulated ZGEMM
def check_zgemm(C, A, B, s, ta, tb, alpha, beta, C0):
    E = oracle.zgemm_emu(A, B, s, ta, tb, alpha, beta, C0)
    opA = A if ta == "N" else (A.T if ta == "T" else A.conj().T)
    opB = B if tb == "N" else (B.T if tb == "T" else B.conj().T)
    AB = (np.abs(opA.real) + np.abs(opA.imag)) @ (np.abs(opB.real) + np.abs(opB.imag))
    tol = 8 * (s + 2) * U * abs(alpha) * AB + 4 * U * np.abs(E)
    if C0 is not None and beta != 0:
        tol = tol + 4 * U * abs(beta) * np.abs(C0)
    assert (np.abs(C.real - E.real) <= tol).all()
    assert (np.abs(C.imag - E.imag) <= tol).all()


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("C", "N"), ("T", "C"), ("N", "T"), ("C", "C")])
@pytest.mark.parametrize("m,n,k,s", [(64, 128, 96, 7), (77, 150, 333, 4), (3, 5, 2, 9)])
def test_zgemm_parity(ozg, ctx, ta, tb, m, n, k, s):
    shA = (m, k) if ta == "N" else (k, m)
    shB = (k, n) if tb == "N" else (n, k)
    A = wide(shA, 1.5, m + k) + 1j * wide(shA, 1.5, m + k + 1)
    B = wide(shB, 1.5, n + k) + 1j * wide(shB, 1.5, n + k + 1)
    C = torch.zeros((n, m), dtype=torch.complex128, device="cuda")
    ctx.zgemm(ta, tb, m, n, k, 1.0, dev(ozg, A), A.shape[0], dev(ozg, B), B.shape[0], 0.0, C, m, s)
    ctx.sync()
    check_zgemm(host(ozg, C, m, n), A, B, s, ta, tb, 1.0, 0.0, None)


def test_zgemm_alpha_beta(ozg, ctx):
    m, n, k, s = 90, 70, 50, 8
    A, B = workloads.kkr_like_pair(nblk=3, bs=32, seed=71)
    A, B = np.asfortranarray(A[:m, :k]), np.asfortranarray(B[:k, :n])
    C0 = np.asfortranarray(workloads.rng(72).normal(size=(m, n)) + 1j * workloads.rng(73).normal(size=(m, n)))
    al, be = 0.5 - 2j, 1.5 + 0.25j
    dC = dev(ozg, C0)
    ctx.zgemm("N", "N", m, n, k, al, dev(ozg, A), m, dev(ozg, B), k, be, dC, m, s)
    ctx.sync()
    check_zgemm(host(ozg, dC, m, n), A, B, s, "N", "N", al, be, C0)


# ----------------------------------------------------------------------------- native FP64
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "T"), ("N", "T")])
def test_native_dgemm(ozg, ctx, ta, tb):
    m, n, k = 131, 77, 203
    A = wide((m, k) if ta == "N" else (k, m), 2.0, 81)
    B = wide((k, n) if tb == "N" else (n, k), 2.0, 82)
    C0 = np.asfortranarray(workloads.rng(83).normal(size=(m, n)))
    dC = dev(ozg, C0)
    ctx.native_dgemm(ta, tb, m, n, k, 1.5, dev(ozg, A), A.shape[0], dev(ozg, B), B.shape[0], -0.5, dC, m)
    ctx.sync()
    C = host(ozg, dC, m, n)
    hi, lo = oracle.dgemm_dd(A, B, ta, tb, 1.5, -0.5, C0)
    AB = oracle.abs_product(A, B, ta, tb)
    gk = (k + 2) * U / (1 - (k + 2) * U)
    assert (np.abs(C - hi - lo) <= gk * (1.5 * AB + 0.5 * np.abs(C0)) + 2 * U * np.abs(hi)).all()


def test_native_zgemm_and_slices_minus_one(ozg, ctx):
    m, n, k = 40, 33, 65
    A = wide((k, m), 1.0, 91) + 1j * wide((k, m), 1.0, 92)
    B = wide((k, n), 1.0, 93) + 1j * wide((k, n), 1.0, 94)
    dC = torch.zeros((n, m), dtype=torch.complex128, device="cuda")
    ctx.zgemm("C", "N", m, n, k, 1.0, dev(ozg, A), k, dev(ozg, B), k, 0.0, dC, m, -1)
    ctx.sync()
    C = host(ozg, dC, m, n)
    ref = A.conj().T @ B
    np.testing.assert_allclose(C, ref, rtol=0, atol=4 * k * U * np.abs(ref).max() + 1e-15)


# ----------------------------------------------------------------------------- full size, sampled
def test_full_size_dgemm_sampled(ozg, ctx):
    """The 8192^3 wide-exponent DGEMM in the benchmark's launch configuration (256-wide tiles with
    deferred pushes); sampled rows and columns equal the oracle's emulation bit for bit (per-row
    and per-column scales make the sampled block's emulation identical to the full one's)."""
    m = n = k = 8192
    s = 7
    A, B = workloads.wide_exponent_pair(m, n, k, 0.5, seed=2)
    dA, dB = dev(ozg, A), dev(ozg, B)
    dC = torch.zeros((n, m), dtype=torch.float64, device="cuda")
    ctx.dgemm("N", "N", m, n, k, 1.0, dA, m, dB, k, 0.0, dC, m, s)
    ctx.sync()
    g = workloads.rng(99)
    rows = np.sort(g.choice(m, 24, replace=False))
    cols = np.sort(g.choice(n, 24, replace=False))
    rows = np.concatenate([rows, [0, m - 1]])
    cols = np.concatenate([cols, [0, n - 1]])
    Cs = dC.cpu().numpy().T[np.ix_(rows, cols)]
    As = np.asfortranarray(A[rows])
    Bs = np.asfortranarray(B[:, cols])
    assert windows(s, k) <= 2  # two exact windows: the oracle's definition bit for bit
    assert np.array_equal(Cs, oracle.dgemm_emu(As, Bs, s))


# ----------------------------------------------------------------------------- sampled dd check
@pytest.mark.parametrize("s", [3, 5, 8])
def test_sampled_check_estimate(ozg, ctx, s):
    """The GPU double-double check reports the error of sampled entries: never above the true
    maximum over all entries (oracle), and of the same order (errors are homogeneous here)."""
    m, n, k = 160, 300, 700
    A, B = workloads.wide_exponent_pair(m, n, k, 1.0, seed=101)
    dC = torch.zeros((n, m), dtype=torch.float64, device="cuda")
    ctx.set_check_samples(256)
    try:
        rep = ctx.dgemm("N", "N", m, n, k, 1.0, dev(ozg, A), m, dev(ozg, B), k, 0.0, dC, m, s, report=True)
    finally:
        ctx.set_check_samples(0)
    full = oracle.rel_err_vs_dd(host(ozg, dC, m, n), A, B)
    assert rep.samples == 256
    assert rep.est_err <= full * (1 + 1e-9) + 1e-300
    assert rep.est_err >= full / 50


def test_sampled_check_beta_and_complex(ozg, ctx):
    m, n, k, s = 70, 90, 120, 4
    A = wide((m, k), 1.0, 111) + 1j * wide((m, k), 1.0, 112)
    B = wide((k, n), 1.0, 113) + 1j * wide((k, n), 1.0, 114)
    C0 = np.asfortranarray(workloads.rng(115).normal(size=(m, n)) + 1j * workloads.rng(116).normal(size=(m, n)))
    dC = dev(ozg, C0)
    ctx.set_check_samples(128)
    try:
        rep = ctx.zgemm("N", "N", m, n, k, 0.5 + 1j, dev(ozg, A), m, dev(ozg, B), k, -1.0 + 0.5j, dC, m, s,
                        report=True)
        assert rep.samples == 128 and 0 < rep.est_err < 1e-5
        # real, beta != 0
        Ar, Br = A.real.copy(order="F"), B.real.copy(order="F")
        C0r = np.asfortranarray(C0.real)
        dCr = dev(ozg, C0r)
        rep = ctx.dgemm("N", "N", m, n, k, 2.0, dev(ozg, Ar), m, dev(ozg, Br), k, 0.5, dCr, m, s, report=True)
        Cg = host(ozg, dCr, m, n)
        full = oracle.rel_err_vs_dd(Cg, Ar, Br, alpha=2.0, beta=0.5, C0=C0r)
        assert 0 < rep.est_err <= full * (1 + 1e-9)
    finally:
        ctx.set_check_samples(0)


# ----------------------------------------------------------------------------- exact epilogue
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "T")])
@pytest.mark.parametrize("m,n,k,s", [(200, 300, 500, 7), (129, 257, 1100, 13), (64, 64, 64, 3), (5, 3, 2000, 10)])
def test_dgemm_bit_exact_single_rounding(ozg, ctx, ta, tb, m, n, k, s):
    """In the opt-in correctly rounded mode (s <= 13) the epilogue sums the group products
    exactly (128-bit Horner) and rounds once: with alpha = 1, beta = 0 the result equals the
    oracle's definition bit for bit, also where the default mode needs a third window."""
    A = wide((m, k) if ta == "N" else (k, m), 2.0, 7 * m + k)
    B = wide((k, n) if tb == "N" else (n, k), 2.0, 5 * n + k)
    C = torch.zeros((n, m), dtype=torch.float64, device="cuda")
    ctx.set_exact_epilogue(True)
    try:
        ctx.dgemm(ta, tb, m, n, k, 1.0, dev(ozg, A), A.shape[0], dev(ozg, B), B.shape[0], 0.0, C, m, s)
        ctx.sync()
    finally:
        ctx.set_exact_epilogue(False)
    assert np.array_equal(host(ozg, C, m, n), oracle.dgemm_emu(A, B, s, ta, tb))


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("C", "T")])
def test_zgemm_bit_exact_single_rounding(ozg, ctx, ta, tb):
    m, n, k, s = 70, 90, 300, 9
    shA = (m, k) if ta == "N" else (k, m)
    shB = (k, n) if tb == "N" else (n, k)
    A = wide(shA, 1.0, 801) + 1j * wide(shA, 1.0, 802)
    B = wide(shB, 1.0, 803) + 1j * wide(shB, 1.0, 804)
    C = torch.zeros((n, m), dtype=torch.complex128, device="cuda")
    ctx.set_exact_epilogue(True)
    try:
        ctx.zgemm(ta, tb, m, n, k, 1.0, dev(ozg, A), A.shape[0], dev(ozg, B), B.shape[0], 0.0, C, m, s)
        ctx.sync()
    finally:
        ctx.set_exact_epilogue(False)
    assert np.array_equal(host(ozg, C, m, n), oracle.zgemm_emu(A, B, s, ta, tb))


def windows(s, k, cplx=False):
    """Number of exact int64 windows the default epilogue uses: the largest group count c with
    (s k_pad 127^2 [x2 complex]) 128^(c-1) 128/127 < 2^63, and ceil(s / c) windows."""
    gmax = s * (-(-k // 64) * 64) * 127 * 127 * (2 if cplx else 1)
    c = max(1, (62 - gmax.bit_length()) // 7 + 1)
    return -(-s // c)


@pytest.mark.parametrize("ta,tb,m,n,k,s,alpha,beta", [
    ("N", "N", 200, 300, 500, 7, 1.0, 0.0),
    ("T", "N", 77, 50, 300, 12, 1.0, 0.0),
    ("N", "T", 300, 130, 8200, 7, -0.5, 0.25),   # long k: chains and pushes split a group
    ("T", "T", 5, 3, 2000, 10, 3.0, 1.0),
    ("N", "N", 129, 257, 64, 3, 1.0, 0.0),
])
def test_dgemm_default_bit_exact_two_windows(ozg, ctx, ta, tb, m, n, k, s, alpha, beta):
    """With at most two int64 windows the default epilogue sums the group products exactly and
    rounds once (integer instructions), so it equals the oracle's definition bit for bit, alpha
    and beta included (same fma order)."""
    assert windows(s, k) <= 2
    A = wide((m, k) if ta == "N" else (k, m), 2.0, 3 * m + k)
    B = wide((k, n) if tb == "N" else (n, k), 2.0, 3 * n + k)
    C0 = np.asfortranarray(workloads.rng(m + n).uniform(-1, 1, (m, n)))
    C = dev(ozg, C0)
    ctx.dgemm(ta, tb, m, n, k, alpha, dev(ozg, A), A.shape[0], dev(ozg, B), B.shape[0], beta, C, m, s)
    ctx.sync()
    assert np.array_equal(host(ozg, C, m, n), oracle.dgemm_emu(A, B, s, ta, tb, alpha, beta, C0))


@pytest.mark.parametrize("ta,tb,alpha,beta", [("N", "N", 1.0, 0.0), ("C", "T", 0.5 - 2j, 1.5 + 0.25j)])
def test_zgemm_default_bit_exact_two_windows(ozg, ctx, ta, tb, alpha, beta):
    m, n, k, s = 70, 90, 300, 9
    assert windows(s, k, cplx=True) <= 2
    shA = (m, k) if ta == "N" else (k, m)
    shB = (k, n) if tb == "N" else (n, k)
    A = wide(shA, 1.0, 821) + 1j * wide(shA, 1.0, 822)
    B = wide(shB, 1.0, 823) + 1j * wide(shB, 1.0, 824)
    C0 = np.asfortranarray(workloads.rng(825).normal(size=(m, n)) + 1j * workloads.rng(826).normal(size=(m, n)))
    C = dev(ozg, C0)
    ctx.zgemm(ta, tb, m, n, k, alpha, dev(ozg, A), A.shape[0], dev(ozg, B), B.shape[0], beta, C, m, s)
    ctx.sync()
    assert np.array_equal(host(ozg, C, m, n), oracle.zgemm_emu(A, B, s, ta, tb, alpha, beta, C0))


@pytest.mark.parametrize("exact", [False, True])
def test_dgemm_subnormal_and_overflow_results_single_rounding(ozg, ctx, exact):
    """Results below 2^-1022 and past the largest finite value are rounded once, as the oracle
    defines them: onto the grid of the smallest subnormal directly (rounding to 53 bits first
    would take 2^-1075 + 2^-1130 to the tie 2^-1075 and then to 0), or to +-inf; in the default
    (two-window) and in the exact epilogue."""
    cases = [(np.asfortranarray([[2.0 ** -500, 2.0 ** -555]]), np.asfortranarray([[2.0 ** -575], [2.0 ** -575]]), 8)]
    m, n, k = 150, 140, 300
    for scale, seed in ((-540, 1), (510, 2)):
        cases.append((np.asfortranarray(wide((m, k), 2.0, 951 + seed) * 2.0 ** scale),
                      np.asfortranarray(wide((k, n), 2.0, 961 + seed) * 2.0 ** scale), 7))
    ctx.set_exact_epilogue(exact)
    try:
        for i, (A, B, s) in enumerate(cases):
            m_, k_ = A.shape
            n_ = B.shape[1]
            assert windows(s, k_) <= 2
            C = torch.zeros((n_, m_), dtype=torch.float64, device="cuda")
            ctx.dgemm("N", "N", m_, n_, k_, 1.0, dev(ozg, A), m_, dev(ozg, B), k_, 0.0, C, m_, s)
            ctx.sync()
            want = oracle.dgemm_emu(A, B, s)
            if i == 0:
                assert want[0, 0] == 2.0 ** -1074
            elif i == 1:
                assert ((want != 0) & (np.abs(want) < 2.0 ** -1022)).sum() > 1000
            else:
                assert np.isinf(want).sum() > 100 and np.isfinite(want).sum() > 100
            assert np.array_equal(host(ozg, C, m_, n_), want)
    finally:
        ctx.set_exact_epilogue(False)


@pytest.mark.parametrize("k,s", [(1100, 13), (300, 14), (300, 18), (5000, 16)])
def test_dgemm_three_or_more_windows_fp64(ozg, ctx, k, s):
    """Beyond two windows the partial sum continues in FP64 (one rounding per window): within the
    stated tolerance of the oracle."""
    assert windows(s, k) >= 3
    m, n = 90, 130
    A, B = wide((m, k), 3.0, 831 + k), wide((k, n), 3.0, 832 + k)
    C = torch.zeros((n, m), dtype=torch.float64, device="cuda")
    ctx.dgemm("N", "N", m, n, k, 1.0, dev(ozg, A), m, dev(ozg, B), k, 0.0, C, m, s)
    ctx.sync()
    check_dgemm(host(ozg, C, m, n), A, B, s, "N", "N", 1.0, 0.0, None)


def test_dgemm_s_above_13_fp64_epilogue(ozg, ctx):
    m, n, k = 100, 140, 300
    A, B = wide((m, k), 3.0, 811), wide((k, n), 3.0, 812)
    for s in (14, 18):
        C = torch.zeros((n, m), dtype=torch.float64, device="cuda")
        ctx.dgemm("N", "N", m, n, k, 1.0, dev(ozg, A), m, dev(ozg, B), k, 0.0, C, m, s)
        ctx.sync()
        check_dgemm(host(ozg, C, m, n), A, B, s, "N", "N", 1.0, 0.0, None)


def test_check_reports_paper_part_errors_for_complex(ozg, ctx):
    """max_real / max_imag: per-part error relative to the part (the MuST study's measure), never
    above the maximum over all entries computed by the oracle."""
    m, n, k, s = 60, 50, 200, 5
    A = wide((m, k), 1.0, 901) + 1j * wide((m, k), 1.0, 902)
    B = wide((k, n), 1.0, 903) + 1j * wide((k, n), 1.0, 904)
    dC = torch.zeros((n, m), dtype=torch.complex128, device="cuda")
    ctx.set_check_samples(128)
    try:
        rep = ctx.zgemm("N", "N", m, n, k, 1.0, dev(ozg, A), m, dev(ozg, B), k, 0.0, dC, m, s, report=True)
    finally:
        ctx.set_check_samples(0)
    C = host(ozg, dC, m, n)
    rh, rl, ih, il = oracle.zgemm_dd(A, B)
    full_re = np.max(np.abs(C.real - rh - rl) / np.abs(rh))
    full_im = np.max(np.abs(C.imag - ih - il) / np.abs(ih))
    assert 0 < rep.max_real <= full_re * (1 + 1e-9)
    assert 0 < rep.max_imag <= full_im * (1 + 1e-9)
    assert rep.max_real >= full_re / 1e4 and rep.max_imag >= full_im / 1e4


# ----------------------------------------------------------------------------- 3M ZGEMM
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("C", "N"), ("N", "T"), ("N", "C"), ("C", "T")])
@pytest.mark.parametrize("m,n,k,s", [(70, 90, 300, 7), (5, 3, 2000, 10), (129, 257, 64, 4)])
def test_zgemm3m_bit_exact_vs_oracle(ozg, ctx, ta, tb, m, n, k, s):
    """3M ZGEMM (three real emulated products; Re = RN(P1 - P2), Im = RN(RN(P3 - P1) - P2))
    equals the oracle's 3M definition bit for bit: each real product is the exactly rounded
    emulation (s <= 10), the combine and alpha, beta are the same FP64 operations in the same
    order."""
    shA = (m, k) if ta == "N" else (k, m)
    shB = (k, n) if tb == "N" else (n, k)
    seed = 7 * m + 3 * n + k + ord(ta) + 2 * ord(tb)
    A = wide(shA, 1.5, seed) + 1j * wide(shA, 1.5, seed + 1)
    B = wide(shB, 1.5, seed + 2) + 1j * wide(shB, 1.5, seed + 3)
    C0 = np.asfortranarray(workloads.rng(seed + 4).normal(size=(m, n)) + 1j * workloads.rng(seed + 5).normal(size=(m, n)))
    al, be = 0.5 - 2j, 1.5 + 0.25j
    C = dev(ozg, C0)
    rep = ctx.zgemm3m(ta, tb, m, n, k, al, dev(ozg, A), A.shape[0], dev(ozg, B), B.shape[0], be, C, m, s, report=True)
    ctx.sync()
    assert rep.status == 0 and rep.slices_used == s
    assert np.array_equal(host(ozg, C, m, n), oracle.zgemm3m_emu(A, B, s, ta, tb, al, be, C0))


def test_zgemm3m_check_report_and_arguments(ozg, ctx):
    """The sampled check judges the 3M result: its estimate lies within the 3M bound's scale;
    slices = 0 is rejected (argument 14); native mode and alpha = 0 take the stacked path."""
    m, n, k, s = 60, 50, 400, 7
    A = wide((m, k), 1.0, 901) + 1j * wide((m, k), 1.0, 902)
    B = wide((k, n), 1.0, 903) + 1j * wide((k, n), 1.0, 904)
    ctx.set_check_samples(64)
    try:
        C = dev(ozg, np.zeros((m, n), dtype=np.complex128))
        rep = ctx.zgemm3m("N", "N", m, n, k, 1.0, dev(ozg, A), m, dev(ozg, B), k, 0.0, C, m, s, report=True)
    finally:
        ctx.set_check_samples(0)
    bre, bim = oracle.zgemm3m_bound(A, B, s)
    scale = oracle.abs_product(np.abs(A.real) + np.abs(A.imag), np.abs(B.real) + np.abs(B.imag))
    assert rep.samples == 64 and 0 <= rep.est_err <= max((bre / scale).max(), (bim / scale).max()) * 4
    assert np.isfinite(rep.max_real) and np.isfinite(rep.max_imag)
    dA, dB = dev(ozg, A), dev(ozg, B)
    rc = ozg.load().ozg_zgemm3m(ctx._h, b"N", b"N", m, n, k, (ctypes_d2(1.0, 0.0)), dA.data_ptr(), m, dB.data_ptr(), k,
                                (ctypes_d2(0.0, 0.0)), C.data_ptr(), m, 0, None)
    assert rc == -14
    Cn = dev(ozg, np.zeros((m, n), dtype=np.complex128))
    ctx.zgemm3m("N", "N", m, n, k, 1.0, dA, m, dB, k, 0.0, Cn, m, -1)
    ctx.sync()
    np.testing.assert_allclose(host(ozg, Cn, m, n), A @ B, rtol=0, atol=(k + 2) * 4 * U * scale.max())


def ctypes_d2(re, im):
    import ctypes
    return (ctypes.c_double * 2)(re, im)


def test_zgemm3m_padded_leading_dimensions(ozg, ctx):
    """3M with lda, ldb, ldc above the matrix heights (the deinterleave and combine kernels do
    their own leading-dimension arithmetic): bit-equal to the oracle on the op'd matrices, C's
    padding rows untouched."""
    m, n, k, s = 37, 29, 53, 8
    g = workloads.rng(930)
    opA = wide((m, k), 1.0, 931) + 1j * wide((m, k), 1.0, 932)
    opB = wide((k, n), 1.0, 933) + 1j * wide((k, n), 1.0, 934)
    lda, ldb, ldc = k + 4, k + 1, m + 3
    A = np.zeros((lda, m), dtype=np.complex128, order="F")
    A[:k] = opA.T                                  # op = 'T'
    B = np.zeros((ldb, n), dtype=np.complex128, order="F")
    B[:k] = opB                                    # op = 'N'
    C0 = np.asfortranarray(g.normal(size=(ldc, n)) + 1j * g.normal(size=(ldc, n)))
    C = dev(ozg, C0)
    ctx.zgemm3m("T", "N", m, n, k, 1.25 - 0.5j, dev(ozg, A), lda, dev(ozg, B), ldb, -0.5 + 1j, C, ldc, s)
    ctx.sync()
    out = host(ozg, C, ldc, n)
    assert np.array_equal(out[m:], C0[m:])
    E = oracle.zgemm3m_emu(np.asfortranarray(opA), np.asfortranarray(opB), s, "N", "N", 1.25 - 0.5j, -0.5 + 1j,
                           np.asfortranarray(C0[:m]))
    assert np.array_equal(out[:m], E)
