"""ozg_dgemm_noalloc: the emulated DGEMM for callers that cannot allocate device memory (an
interposed dgemm_ in an application that owns all device memory through its own pool or budget,
latency-critical paths where cudaMalloc would synchronise the device).  It keeps its scratch in a
fixed in-library device array.  These tests call it through the C ABI and compare it with
ozg_dgemm on two calls in a row, bit for bit (both sum every group exactly and round once at
these slice counts), and with the oracle's emulation.  A third call is large enough that the
array holds fewer CTA tiles than the output has, so each CTA loops over several tiles.  This file
is collected last on purpose."""
import numpy as np
import pytest

import oracle
from paper_2503_22875_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCRATCH = 64 << 20          # OZG_NOALLOC_SCRATCH_BYTES
TILE = 128 * 256 * 16       # OZG_NOALLOC_TILE_BYTES


@pytest.fixture(scope="module")
def ozg():
    from paper_2503_22875_gb300 import build, ozg
    build.build()
    ozg.load()
    return ozg


def band_samples(total, band, g):
    idx = {0, total - 1}
    for b0 in range(0, total, band):
        idx.add(int(g.integers(b0, min(total, b0 + band))))
    return np.array(sorted(idx))


def scratch_ctas(m, n, k, s):
    """CTAs the array leaves room for (the carve of ozg_noalloc.cu, each part rounded to 256)."""
    r = lambda x: (x + 255) // 256 * 256  # noqa: E731
    kp = (k + 7) // 8 * 8
    off = r(16) + r(8 * m) + r(8 * n) + r(4 * m) + r(4 * n) + r(2 * s * m * kp) + r(2 * s * n * kp)
    return (SCRATCH - off) // TILE


CASES = [(300, 520, 700, 7, "N", "N", 1.0, 0.0),
         (1000, 900, 1100, 6, "T", "N", -0.5, 0.75),
         (2048, 2048, 256, 8, "N", "T", 2.0, 0.0)]   # scratch for 95 CTAs, 128 output tiles


def test_noalloc_matches_dgemm_and_oracle_on_consecutive_calls(ozg):
    assert scratch_ctas(2048, 2048, 256, 8) < (2048 // 128) * (2048 // 256)
    ctx = ozg.Context()
    free_after = []
    for m, n, k, s, ta, tb, alpha, beta in CASES:
        A, B = workloads.wide_exponent_pair(m, n, k, 1.0, seed=m + n + k)
        A = np.asfortranarray(A.T) if ta == "T" else A
        B = np.asfortranarray(B.T) if tb == "T" else B
        C0 = np.asfortranarray(workloads.rng(k).uniform(-1, 1, (m, n)))
        dA, dB = ozg.to_device(A), ozg.to_device(B)
        C_ref, C_na = ozg.to_device(C0), ozg.to_device(C0)
        torch.cuda.synchronize()
        ctx.dgemm(ta, tb, m, n, k, alpha, dA, A.shape[0], dB, B.shape[0], beta, C_ref, m, s)
        ctx.sync()
        f0 = torch.cuda.mem_get_info()[0]
        rc = ozg.dgemm_noalloc(ta, tb, m, n, k, alpha, dA, A.shape[0], dB, B.shape[0], beta, C_na, m, s)
        torch.cuda.synchronize()
        assert rc == 0, ozg.strerror(rc)
        free_after.append((f0, torch.cuda.mem_get_info()[0]))
        R = ozg.from_device(C_ref, m, n)
        X = ozg.from_device(C_na, m, n)
        assert np.array_equal(X, R), (m, n, k, s)
        # against the oracle on one row / column in every 128-row / 128-column band (per-row and
        # per-column scales make the block's emulation the full product's on those entries)
        g = workloads.rng(m * n)
        rows, cols = band_samples(m, 128, g), band_samples(n, 128, g)
        opA = A.T if ta == "T" else A
        opB = B.T if tb == "T" else B
        E = oracle.dgemm_emu(np.asfortranarray(opA[rows]), np.asfortranarray(opB[:, cols]), s, "N", "N", alpha, beta,
                             np.asfortranarray(C0[np.ix_(rows, cols)]))
        assert np.array_equal(X[np.ix_(rows, cols)], E), (m, n, k, s)
    # the later calls allocated nothing on the device
    for f0, f1 in free_after[1:]:
        assert f1 >= f0
    ctx.close()


def test_noalloc_rejects_problems_beyond_its_scratch(ozg):
    big = 4096  # digit planes alone need ~470 MB at s = 7
    rc = ozg.dgemm_noalloc("N", "N", big, big, big, 1.0, 0, big, 0, big, 0.0, 0, big, 7)
    assert rc == 4  # OZG_ERR_UNSUPPORTED, before any work is queued
    assert ozg.dgemm_noalloc("N", "N", 4, 4, 4, 1.0, 0, 3, 0, 4, 0.0, 0, 4, 7) == -8
    assert ozg.dgemm_noalloc("N", "N", 4, 4, 4, 1.0, 0, 4, 0, 4, 0.0, 0, 4, 0) == -14
