"""Fault paths without a GPU fault: a bounded device-side wait that runs out reports
OZG_ERR_TIMEOUT through ozg_sync and leaves the context usable; an injected workspace
allocation failure returns OZG_ERR_ALLOC with C untouched, and the next call allocates again."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2503_22875_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
OZG_ERR_ALLOC, OZG_ERR_TIMEOUT = 2, 3


@pytest.fixture(scope="module")
def ozg():
    from paper_2503_22875_gb300 import build, ozg
    build.build()
    ozg.load()
    return ozg


def small_dgemm(ozg, L, ctx, seed):
    m, n, k = 70, 90, 130
    A, B = workloads.wide_exponent_pair(m, n, k, 1.0, seed=seed)
    C0 = np.asfortranarray(workloads.rng(seed + 1).uniform(-1, 1, (m, n)))
    dA, dB, dC = ozg.to_device(A), ozg.to_device(B), ozg.to_device(C0)
    rc = L.ozg_dgemm(ctx._h, b"N", b"N", m, n, k, 0.5, dA.data_ptr(), m, dB.data_ptr(), k, 0.25, dC.data_ptr(), m, 7,
                     None)
    return rc, ozg.from_device(dC, m, n), oracle.dgemm_emu(A, B, 7, "N", "N", 0.5, 0.25, C0), C0


def test_bounded_wait_times_out_and_context_survives(ozg):
    L = ozg.load()
    ctx = ozg.Context()
    assert L.ozg_debug_wait(ctx._h, 10) == 5  # limit outside 1000 .. 4e9
    assert L.ozg_debug_wait(ctx._h, 20_000_000) == 0  # ~10 ms
    assert L.ozg_sync(ctx._h) == OZG_ERR_TIMEOUT
    assert L.ozg_sync(ctx._h) == 0  # reported once
    rc, C, E, _ = small_dgemm(ozg, L, ctx, 701)
    assert rc == 0 and L.ozg_sync(ctx._h) == 0
    assert np.array_equal(C, E)
    ctx.close()


def test_workspace_allocation_failure_reported_and_recovered(ozg):
    L = ozg.load()
    ctx = ozg.Context()
    assert L.ozg_debug_fail_allocs(ctx._h, 1) == 0
    rc, C, _, C0 = small_dgemm(ozg, L, ctx, 711)
    assert rc == OZG_ERR_ALLOC
    assert np.array_equal(C, C0)  # C untouched
    rc, C, E, _ = small_dgemm(ozg, L, ctx, 711)
    assert rc == 0 and L.ozg_sync(ctx._h) == 0 and np.array_equal(C, E)
    # grouped calls: their own workspace
    batch = [workloads.wide_exponent_pair(40 + 9 * i, 30 + 7 * i, 50 + 11 * i, 1.0, seed=720 + i) for i in range(4)]
    dev = [(ozg.to_device(A), ozg.to_device(B), torch.zeros((B.shape[1], A.shape[0]), dtype=torch.float64,
                                                              device="cuda")) for A, B in batch]
    descs = (ozg.GemmDesc * 4)()
    for i, ((A, B), (dA, dB, dC)) in enumerate(zip(batch, dev)):
        m, k, n = A.shape[0], A.shape[1], B.shape[1]
        descs[i] = ozg.GemmDesc(b"N", b"N", b"", m, n, k, 1.0, 0.0, dA.data_ptr(), m, dB.data_ptr(), k, dC.data_ptr(), m)
    sl = (ctypes.c_int * 4)(5, 6, 7, 8)
    assert L.ozg_debug_fail_allocs(ctx._h, 1) == 0
    assert L.ozg_dgemm_grouped(ctx._h, 4, descs, sl, None) == OZG_ERR_ALLOC
    assert all(float(torch.abs(d[2]).max()) == 0.0 for d in dev)
    assert L.ozg_dgemm_grouped(ctx._h, 4, descs, sl, None) == 0 and L.ozg_sync(ctx._h) == 0
    for (A, B), (_, _, dC), s in zip(batch, dev, (5, 6, 7, 8)):
        assert np.array_equal(ozg.from_device(dC, A.shape[0], B.shape[1]), oracle.dgemm_emu(A, B, s))
    ctx.close()
