"""ozg_dgemm_noalloc: the emulated DGEMM for callers that cannot allocate device memory (code
running under CUDA-graph stream capture, an interposed dgemm_ in an application that owns all
device memory, latency-critical paths where cudaMalloc would synchronise the device).  It keeps
its scratch in a fixed in-library device array; these tests call it through the C ABI and
compare it with ozg_dgemm on two calls in a row.  This file is collected last on purpose."""
import numpy as np
import pytest

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


def test_noalloc_matches_dgemm_on_two_calls(ozg):
    ctx = ozg.Context()
    cases = [(300, 520, 700, 7, "N", "N", 1.0, 0.0), (1000, 900, 1100, 6, "T", "N", -0.5, 0.75)]
    free_after = []
    for m, n, k, s, ta, tb, alpha, beta in cases:
        A, B = workloads.wide_exponent_pair(m, n, k, 1.0, seed=m + n + k)
        A = np.asfortranarray(A.T) if ta == "T" else A
        C0 = np.asfortranarray(workloads.rng(k).uniform(-1, 1, (m, n)))
        dA, dB = ozg.to_device(A), ozg.to_device(B)
        C_ref, C_na = ozg.to_device(C0), ozg.to_device(C0)
        torch.cuda.synchronize()
        ctx.dgemm(ta, tb, m, n, k, alpha, dA, A.shape[0], dB, k, beta, C_ref, m, s)
        ctx.sync()
        f0 = torch.cuda.mem_get_info()[0]
        rc = ozg.dgemm_noalloc(ta, tb, m, n, k, alpha, dA, A.shape[0], dB, k, beta, C_na, m, s)
        torch.cuda.synchronize()
        assert rc == 0, ozg.strerror(rc)
        free_after.append((f0, torch.cuda.mem_get_info()[0]))
        R = ozg.from_device(C_ref, m, n)
        X = ozg.from_device(C_na, m, n)
        opA = A.T if ta == "T" else A
        AB = np.abs(opA) @ np.abs(B)
        tol = 4 * (s + 2) * U * abs(alpha) * AB + 2 * U * np.abs(R) + 2 * U * abs(beta) * np.abs(C0)
        assert (np.abs(X - R) <= tol).all()
    # the second call allocated nothing on the device
    f0, f1 = free_after[1]
    assert f1 >= f0
    ctx.close()


def test_noalloc_rejects_problems_beyond_its_scratch(ozg):
    big = 4096  # digit planes alone need ~470 MB at s = 7
    rc = ozg.dgemm_noalloc("N", "N", big, big, big, 1.0, 0, big, 0, big, 0.0, 0, big, 7)
    assert rc == 4  # OZG_ERR_UNSUPPORTED, before any work is queued
    assert ozg.dgemm_noalloc("N", "N", 4, 4, 4, 1.0, 0, 3, 0, 4, 0.0, 0, 4, 7) == -8
    assert ozg.dgemm_noalloc("N", "N", 4, 4, 4, 1.0, 0, 4, 0, 4, 0.0, 0, 4, 0) == -14
