"""Learned slice selector on the GPU: features, gradients and decisions against the oracle, the
automatic path (selection, check, re-run at the fallback count) against the emulation oracle,
and the labels of the training data against the oracle's double-double errors."""
import numpy as np
import pytest

import oracle
from paper_2503_22875_gb300 import selector, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module")
def ozg():
    from paper_2503_22875_gb300 import build, ozg
    build.build()
    ozg.load()
    return ozg


def wide(shape, phi, seed):
    X = workloads.wide_exponent(shape, phi, workloads.rng(seed))
    X.flat[::13] = 0.0
    return np.asfortranarray(X)


@pytest.mark.parametrize("ta,tb,phi", [("N", "N", 3.0), ("T", "N", 6.0), ("N", "T", 0.5), ("T", "T", 2.0)])
def test_features_match_oracle(ozg, ta, tb, phi):
    m, n, k = 150, 90, 333
    A = wide((m, k) if ta == "N" else (k, m), phi, 401)
    B = wide((k, n) if tb == "N" else (n, k), phi, 402)
    ctx = ozg.Context()
    ctx.set_target_error(1e-11)
    f = torch.zeros(24, dtype=torch.float32, device="cuda")
    ctx.selector_features(ta, tb, m, n, k, ozg.to_device(A), A.shape[0], ozg.to_device(B), B.shape[0], f)
    g = f.cpu().numpy()
    o = oracle.features(A, B, 1e-11, ta, tb)
    np.testing.assert_array_equal(g[3:23], o[3:23])
    np.testing.assert_allclose(g[[0, 1, 2, 23]], o[[0, 1, 2, 23]], rtol=1e-6)
    ctx.close()


@pytest.mark.parametrize("ta,tb,m,n,k", [("N", "N", 1, 1, 1), ("N", "N", 17, 9, 2048), ("T", "T", 33, 65, 2049),
                                         ("N", "T", 200, 3, 17), ("T", "N", 16, 8, 1500), ("N", "N", 1000, 700, 100),
                                         ("T", "T", 999, 333, 37)])
def test_features_edges_match_oracle(ozg, ta, tb, m, n, k):
    """Rows of k <= 2048 take the fused statistics kernel (row maxima and gap histogram in one
    read, whole rows per CTA; short rows several row blocks per CTA, the last unit partial),
    longer rows the two-pass kernels: ragged row blocks, an all-zero
    row, runs of zeros longer than a 16-element chunk, subnormal entries, a row scaled below
    2^-987 (whose chunks take the kernel's exact path) and gaps across the 36-exponent edge all
    give the oracle's histogram counts exactly."""
    g = workloads.rng(m * 7 + n * 3 + k)
    opA = workloads.wide_exponent((m, k), 4.0, g)
    opB = workloads.wide_exponent((k, n), 4.0, g)
    if m > 2:
        opA[1, :] = 0.0
        opA[2, : min(k, 40)] = 0.0
        opA[2, -1] = 2.0 ** -1070
        opA[2, 0] = 3.0
        opA[0, : min(k, 5)] = [2.0 ** -e for e in (0, 33, 35, 36, 37)][: min(k, 5)]
    if m > 3:
        opA[3, :] *= 2.0 ** -1000  # maxima below 2^-987 and subnormal entries: the exact path
    if k > 3:
        opB[:3, 0] = [5e-324, 2.0 ** -1022, 1.0]
    A = np.asfortranarray(opA if ta == "N" else opA.T)
    B = np.asfortranarray(opB if tb == "N" else opB.T)
    ctx = ozg.Context()
    f = torch.zeros(24, dtype=torch.float32, device="cuda")
    ctx.selector_features(ta, tb, m, n, k, ozg.to_device(A), A.shape[0], ozg.to_device(B), B.shape[0], f)
    o = oracle.features(A, B, 1e-12, ta, tb)
    np.testing.assert_array_equal(f.cpu().numpy()[3:23], o[3:23])
    ctx.close()


def test_gradients_match_oracle(ozg):
    r = np.random.default_rng(410)
    theta = (r.normal(0, 0.2, selector.PARAMS)).astype(np.float32)
    X = r.normal(size=(200, 24)).astype(np.float32)
    y = r.integers(0, 11, 200).astype(np.int32)
    ctx = ozg.Context()
    ctx.selector_set_params(theta)
    loss, g = ctx.selector_grads(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), 200)
    lo, go = oracle.mlp_loss_grad(theta, X, y)
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
    ctx.close()


def test_training_reduces_loss(ozg):
    r = np.random.default_rng(411)
    X = r.normal(size=(2048, 24)).astype(np.float32)
    w = r.normal(size=(24, 11))
    y = (X @ w).argmax(1).astype(np.int32)  # a learnable rule
    ctx = ozg.Context()
    theta, mean, std, losses = selector.train(ctx, X, y, epochs=30, batch=256, lr=3e-3)
    assert losses[-1] < 0.5 * losses[0]
    ctx.close()


def random_model(path, seed, thr=0.9, fallback=10, bias=None):
    r = np.random.default_rng(seed)
    theta = r.normal(0, 0.3, selector.PARAMS).astype(np.float32)
    if bias is not None:  # force one class: zero last-layer weights, large bias on that class
        p = selector.split_theta(theta)
        theta[selector.PARAMS - 11 - 11 * 64:selector.PARAMS - 11] = 0.0
        theta[selector.PARAMS - 11:] = -20.0
        theta[selector.PARAMS - 11 + bias] = 20.0
    mean = r.normal(size=24).astype(np.float32)
    std = np.abs(r.normal(size=24)).astype(np.float32) + 0.5
    selector.write_model(str(path), theta, mean, std, thr, fallback)
    return selector.read_model(str(path))


def test_decision_matches_cpu_emulation(ozg, tmp_path):
    path = tmp_path / "rand.ozgsel"
    model = random_model(path, 420)
    ctx = ozg.Context()
    ctx.load_selector(str(path))
    f = torch.zeros(24, dtype=torch.float32, device="cuda")
    p = torch.zeros(11, dtype=torch.float32, device="cuda")
    sdev = torch.zeros(1, dtype=torch.int32, device="cuda")
    agree = 0
    for i, phi in enumerate(np.linspace(0, 6, 12)):
        m, n, k = 40 + 17 * i, 70 + 5 * i, 100 + 31 * i
        A, B = wide((m, k), phi, 500 + i), wide((k, n), phi, 600 + i)
        ctx.selector_features("N", "N", m, n, k, ozg.to_device(A), m, ozg.to_device(B), k, f, p, sdev)
        s_cpu, probs = oracle.mlp_select(model, f.cpu().numpy(), 12)
        np.testing.assert_allclose(p.cpu().numpy(), probs, rtol=1e-5, atol=1e-7)
        cum = np.cumsum(probs)
        near = np.any(np.abs(cum - model["thr"]) < 1e-5)
        assert int(sdev.item()) == s_cpu or near
        agree += int(sdev.item()) == s_cpu
    assert agree >= 11
    ctx.close()


def emu_check(ozg, C, A, B, s, alpha=1.0, beta=0.0, C0=None):
    E = oracle.dgemm_emu(A, B, s, "N", "N", alpha, beta, C0)
    tol = 4 * (s + 2) * U * abs(alpha) * oracle.abs_product(A, B) + 2 * U * np.abs(E)
    if C0 is not None:
        tol = tol + 2 * U * abs(beta) * np.abs(C0)
    assert (np.abs(C - E) <= tol).all()


@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_auto_single_call_select_and_repair(ozg, tmp_path, beta):
    m, n, k = 130, 260, 200
    A, B = workloads.wide_exponent_pair(m, n, k, 1.0, seed=430)
    C0 = np.asfortranarray(workloads.rng(431).uniform(-1, 1, (m, n)))
    for bias, expect_repair in ((0, True), (10, False)):  # s = 2 (too small) or s = 12
        path = tmp_path / f"bias{bias}.ozgsel"
        random_model(path, 440 + bias, fallback=9, bias=bias)
        ctx = ozg.Context()
        ctx.load_selector(str(path))
        ctx.set_fallback_slices(9)
        dC = ozg.to_device(C0)
        rep = ctx.dgemm("N", "N", m, n, k, 1.0, ozg.to_device(A), m, ozg.to_device(B), k, beta, dC, m, 0, report=True)
        assert rep.selected == 2 + bias and rep.repaired == int(expect_repair)
        assert rep.slices_used == (9 if expect_repair else 12)
        assert rep.samples >= 64 and rep.est_err <= 1e-12
        emu_check(ozg, ozg.from_device(dC, m, n), A, B, rep.slices_used, 1.0, beta, C0 if beta else None)
        ctx.close()


def test_auto_grouped_mixed(ozg, tmp_path):
    """Learned and fixed calls in one grouped launch, with and without beta: the selector always
    chooses s = 2, so every learned call escalates (s + 2, then the fallback 8); C equals the
    oracle's emulation at the count the call ended with."""
    path = tmp_path / "b0.ozgsel"
    random_model(path, 450, fallback=8, bias=0)  # always s = 2: every automatic call is re-run
    st = torch.cuda.Stream()
    ctx = ozg.Context(stream=st)
    ctx.load_selector(str(path))
    ctx.set_fallback_slices(8)
    batch = []
    for i in range(12):
        m, n, k = 30 + 23 * i, 50 + 11 * i, 40 + 37 * i
        A, B = workloads.wide_exponent_pair(m, n, k, 0.5 * (i % 5), seed=460 + i)
        beta = 0.0 if i % 3 else 1.5
        C0 = np.asfortranarray(workloads.rng(470 + i).uniform(-1, 1, (m, n)))
        s = 0 if i % 2 == 0 else 5
        batch.append((m, n, k, A, B, beta, C0, s, ozg.to_device(A), ozg.to_device(B), ozg.to_device(C0)))
    calls = [("N", "N", m, n, k, 1.0, dA, m, dB, k, beta, dC, m) for (m, n, k, A, B, beta, C0, s, dA, dB, dC) in batch]
    with torch.cuda.stream(st):
        reps = ctx.dgemm_grouped(calls, [b[7] for b in batch], report=True)
    for r, (m, n, k, A, B, beta, C0, s, dA, dB, dC) in zip(reps, batch):
        if s == 0:  # s = 2 is rejected: re-run at 2 + 2 = 4, and when that is rejected too, at 8
            assert r.selected == 2 and r.repaired in (1, 2)
            assert r.slices_used == (4 if r.repaired == 1 else 8)
            assert r.repaired == 2 or r.est_err <= 1e-12
        else:
            assert r.selected == 0 and r.repaired == 0 and r.slices_used == 5
        emu_check(ozg, ozg.from_device(dC, m, n), A, B, r.slices_used, 1.0, beta, C0 if beta else None)
    ctx.close()


def test_training_labels_against_oracle(ozg):
    ctx = ozg.Context()
    X, y, meta = selector.make_dataset(ctx, 6, seed=480, lo=64, hi=200, chunk=3, keep_blocks=True)
    for p, (As, Bs) in enumerate(meta["blocks"]):
        Am = np.asfortranarray(As.T)   # (bm, k)
        Bm = np.asfortranarray(Bs.T)   # (k, bn)
        for ci, s in enumerate(range(2, 13)):
            C = oracle.dgemm_emu(Am, Bm, s)
            full = oracle.rel_err_vs_dd(C, Am, Bm)
            gpu = meta["errs"][p, ci]
            # the sampled estimate is never above the true maximum, up to the epilogue's FP64
            # rounding tolerance (the GPU's C and the oracle's C differ by at most that much)
            assert gpu <= full + 4 * (s + 2) * U
            assert gpu >= full / 100
    ctx.close()


def test_regions_select_per_region_and_match_oracle(ozg):
    """Region-adaptive slice counts: the first band of rows of A has a wide exponent spread and
    the rest a narrow one. Each region's count is the selector's decision on that region's own
    rows of op(A) and columns of op(B) (the oracle's features and MLP). The wide band gets a
    larger count than the narrow ones. Each region meets the target and equals the oracle's
    emulated product at the count it used. Empty bands (more blocks than columns) are quick
    returns."""
    import os
    path = selector.DEFAULT_MODEL
    model = selector.read_model(path)
    s_cap = max(model["s_lo"] + 10, model["fallback"])
    m, n, k = 300, 200, 256
    g = workloads.rng(490)
    A = np.asfortranarray(workloads.wide_exponent((m, k), 0.3, g))
    A[:100] = workloads.wide_exponent((100, k), 5.0, g)
    B = np.asfortranarray(workloads.wide_exponent((k, n), 0.3, g))
    ctx = ozg.Context()
    ctx.load_selector(path)
    ctx.set_target_error(1e-12)
    ctx.set_check_samples(64)
    dC = ozg.to_device(np.zeros((m, n), order="F"))
    reps = ctx.dgemm_regions("N", "N", m, n, k, 1.0, ozg.to_device(A), m, ozg.to_device(B), k, 0.0, dC, m, 3, 2,
                             report=True)
    C = ozg.from_device(dC, m, n)
    sel = {}
    for i in range(3):
        r0, r1 = m * i // 3, m * (i + 1) // 3
        for j in range(2):
            c0, c1 = n * j // 2, n * (j + 1) // 2
            r = reps[i * 2 + j]
            Ai, Bj = np.asfortranarray(A[r0:r1]), np.asfortranarray(B[:, c0:c1])
            s_cpu, probs = oracle.mlp_select(model, oracle.features(Ai, Bj, 1e-12), s_cap)
            near = np.any(np.abs(np.cumsum(probs) - model["thr"]) < 1e-5)
            assert r.selected == s_cpu or near, (i, j, r.selected, s_cpu)
            assert r.status == 0 and r.est_err <= 1e-12
            E = oracle.dgemm_emu(Ai, Bj, r.slices_used)
            if r.slices_used <= 10:  # two exact windows: bit-exact
                assert np.array_equal(C[r0:r1, c0:c1], E), (i, j)
            else:
                emu_check(ozg, C[r0:r1, c0:c1], Ai, Bj, r.slices_used)
            sel[i, j] = r.selected
    assert min(sel[0, 0], sel[0, 1]) > max(sel[2, 0], sel[2, 1])
    # 3 columns cut into 5 bands: [0, 0), [0, 1), [1, 1), [1, 2), [2, 3)
    dC2 = ozg.to_device(np.zeros((m, 3), order="F"))
    reps = ctx.dgemm_regions("N", "N", m, 3, k, 1.0, ozg.to_device(A), m, ozg.to_device(B), k, 0.0, dC2, m, 1, 5,
                             report=True)
    C2 = ozg.from_device(dC2, m, 3)
    assert all(r.status == 0 for r in reps) and reps[0].samples == 0 and reps[2].samples == 0
    for j, col in ((1, 0), (3, 1), (4, 2)):
        Bc = np.asfortranarray(B[:, col:col + 1])
        E = oracle.dgemm_emu(A, Bc, reps[j].slices_used)
        if reps[j].slices_used <= 10:
            assert np.array_equal(C2[:, col:col + 1], E), col
        else:
            emu_check(ozg, C2[:, col:col + 1], A, Bc, reps[j].slices_used)
    ctx.close()


def test_network_gain_over_fixed_counts_in_the_same_pipeline(ozg, tmp_path):
    """What the trained network gains over the method without it.  One 256-call batch of the
    benchmark's distribution (seeded, drawn on the GPU) runs through the identical grouped
    pipeline -- features, the 64-sample check, escalation of rejected calls -- three times: with
    the network's decision, with the constant fallback count (the conservative count the method
    uses without a network) and with each fixed count 8, 9, 10 (rejected calls escalate).  Every
    run meets 1e-12 on every call (sampled check).  The network's run does less tensor work than
    every fixed-count run and is faster than the fallback run."""
    import time
    b = workloads.grouped_batch_flat(256, seed=77)
    calls = b.calls
    descs = b.gemm_calls()
    work = np.array([float(c.m) * c.n * c.k for c in calls])
    st = torch.cuda.Stream()
    fb = selector.read_model(selector.DEFAULT_MODEL)["fallback"]

    def run(model_path):
        ctx = ozg.Context(stream=st)
        ctx.load_selector(model_path)
        ctx.set_target_error(1e-12)
        ctx.set_check_samples(64)
        with torch.cuda.stream(st):
            reps = ctx.dgemm_grouped(descs, [0] * len(descs), report=True)
            torch.cuda.synchronize()
            best = 1e30
            for _ in range(5):
                t0 = time.perf_counter()
                ctx.dgemm_grouped(descs, [0] * len(descs))
                torch.cuda.synchronize()
                best = min(best, time.perf_counter() - t0)
        ctx.close()
        assert all(r.status == 0 and r.est_err <= 1e-12 for r in reps)
        prods = [sum(x * (x + 1) / 2 for x in selector.escalation_passes(r.selected, r.repaired, fb)) for r in reps]
        return best, float(np.dot(prods, work)), reps

    t_net, w_net, reps = run(selector.DEFAULT_MODEL)
    assert len(set(r.selected for r in reps)) >= 3  # the network does choose per call
    fixed = {}
    for s in (8, 9, 10, fb):
        path = str(tmp_path / f"const{s}.ozgsel")
        selector.write_constant_model(path, s, fb)
        fixed[s] = run(path)
        assert all(r.selected == s for r in fixed[s][2])
    for s, (t, w, _) in fixed.items():
        assert w_net < w, (s, w_net / w)
    assert w_net < 0.7 * fixed[fb][1]
    assert t_net < 0.8 * fixed[fb][0], (t_net, fixed[fb][0])


def test_regions_transposed_operands_match_oracle(ozg):
    """Regions over transposed operands (op(A) = A^T, op(B) = B^T, with padded leading
    dimensions): each region equals the oracle's emulation of its own rows of op(A) and columns
    of op(B) at the count it used, and C's padding rows stay untouched."""
    import os
    path = selector.DEFAULT_MODEL
    m, n, k = 150, 110, 90
    g = workloads.rng(495)
    opA = np.asfortranarray(workloads.wide_exponent((m, k), 1.5, g))
    opB = np.asfortranarray(workloads.wide_exponent((k, n), 1.5, g))
    lda, ldb, ldc = k + 3, n + 5, m + 2
    A = np.zeros((lda, m), order="F")
    A[:k] = opA.T
    B = np.zeros((ldb, k), order="F")
    B[:n] = opB.T
    C0 = np.asfortranarray(workloads.rng(496).uniform(-1, 1, (ldc, n)))
    ctx = ozg.Context()
    ctx.load_selector(path)
    ctx.set_target_error(1e-12)
    ctx.set_check_samples(64)
    dC = ozg.to_device(C0)
    reps = ctx.dgemm_regions("T", "T", m, n, k, 0.5, ozg.to_device(A), lda, ozg.to_device(B), ldb, 0.25, dC, ldc,
                             3, 2, report=True)
    C = ozg.from_device(dC, ldc, n)
    assert np.array_equal(C[m:], C0[m:])
    for i in range(3):
        r0, r1 = m * i // 3, m * (i + 1) // 3
        for j in range(2):
            c0, c1 = n * j // 2, n * (j + 1) // 2
            r = reps[i * 2 + j]
            assert r.status == 0 and r.est_err <= 1e-12
            E = oracle.dgemm_emu(np.asfortranarray(opA[r0:r1]), np.asfortranarray(opB[:, c0:c1]), r.slices_used,
                                 "N", "N", 0.5, 0.25, np.asfortranarray(C0[r0:r1, c0:c1]))
            if r.slices_used <= 10:
                assert np.array_equal(C[r0:r1, c0:c1], E), (i, j)
            else:
                emu_check(ozg, C[r0:r1, c0:c1], np.asfortranarray(opA[r0:r1]), np.asfortranarray(opB[:, c0:c1]),
                          r.slices_used, 0.5, 0.25, np.asfortranarray(C0[r0:r1, c0:c1]))
    ctx.close()
