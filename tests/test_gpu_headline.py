"""The learned grouped path of the benchmark headline against the oracle, call by call.

A seeded sample of 64 calls of the headline batch (2048 DGEMMs, m, n, k log-uniform in
[32, 2048], a = (u - 0.5) exp(phi g), phi ~ U(0, 4) per call): the calls with the largest m, n
and k, calls with k in (1024, 2048], and random ones.  They run as one grouped call with
slices = 0 (the selector picks s per call for 1e-12; the sampled check judges every call and
escalates rejected ones: s + 2, then the fallback), on a non-default stream so that the sequence is graph-captured, in the
128-wide tile variant, in the 256-wide one and on CTA pairs (256 x 128 pair tiles).

Per call: the selector's decision equals the oracle's features + MLP decision (up to a
cumulative probability within 1e-5 of the threshold); C equals the oracle's emulation at the
count the call used bit for bit where the epilogue's exact int64 windows cover every group
(two windows: s <= 10 at any k, s <= 12 for k <= 512), else within the stated tolerance of the
FP64 continuation.  Large calls are compared on sampled rows and columns (one row in every
128-row band and one column in every 128-column band, the ragged last ones included): per-row
and per-column scales make the sampled block's emulation identical to the full product's.
"""
import numpy as np
import pytest

import oracle
from paper_2503_22875_gb300 import selector, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U = 2.0 ** -53
TARGET = 1e-12
FULL_COMPARE_MACS = 3e8  # oracle work (m n k s(s+1)/2) below which the whole C is compared


@pytest.fixture(scope="module")
def ozg():
    from paper_2503_22875_gb300 import build, ozg
    build.build()
    ozg.load()
    return ozg


def windows(s, k):
    gmax = s * (-(-k // 64) * 64) * 127 * 127
    c = max(1, (62 - gmax.bit_length()) // 7 + 1)
    return -(-s // c)


def headline_sample(count=64, seed=2025):
    calls = workloads.grouped_batch(2048, seed=4)  # the headline batch's shapes and spreads
    g = workloads.rng(seed)
    pick = {int(np.argmax([c.m for c in calls])), int(np.argmax([c.n for c in calls])),
            int(np.argmax([c.k for c in calls]))}
    long_k = [i for i, c in enumerate(calls) if 1024 < c.k <= 2048]
    pick |= set(int(i) for i in g.choice(long_k, 12, replace=False))
    rest = [i for i in range(len(calls)) if i not in pick]
    pick |= set(int(i) for i in g.choice(rest, count - len(pick), replace=False))
    return [calls[i] for i in sorted(pick)]


def band_samples(total, band, g):
    """One index in every `band`-wide band of range(total), plus the first and the last."""
    idx = {0, total - 1}
    for b0 in range(0, total, band):
        idx.add(int(g.integers(b0, min(total, b0 + band))))
    return np.array(sorted(idx))


@pytest.fixture(scope="module")
def sample():
    out = []
    for c in headline_sample():
        A, B = workloads.call_matrices(c)
        out.append((c, A, B))
    return out


@pytest.mark.parametrize("variant", [1, 5, 0, 4])
def test_learned_grouped_headline_calls_match_oracle(ozg, sample, variant):
    model = selector.read_model(selector.DEFAULT_MODEL)
    s_cap = max(model["s_lo"] + 10, model["fallback"])
    assert max(c.k for c, _, _ in sample) > 1900 and max(c.m for c, _, _ in sample) > 1900
    assert sum(1024 < c.k for c, _, _ in sample) >= 12
    st = torch.cuda.Stream()
    ctx = ozg.Context(stream=st)
    ctx.load_selector(selector.DEFAULT_MODEL)
    ctx.set_target_error(TARGET)
    ctx.set_check_samples(64)
    ctx.set_tile_variant(variant)
    dev = [(ozg.to_device(A), ozg.to_device(B), torch.full((c.n, c.m), np.nan, dtype=torch.float64,
                                                              device="cuda")) for c, A, B in sample]
    calls = [("N", "N", c.m, c.n, c.k, 1.0, dA, c.m, dB, c.k, 0.0, dC, c.m)
             for (c, _, _), (dA, dB, dC) in zip(sample, dev)]
    with torch.cuda.stream(st):
        ctx.dgemm_grouped(calls, [0] * len(calls))           # plan + graph capture
        reps = ctx.dgemm_grouped(calls, [0] * len(calls), report=True)  # graph replay
    g = workloads.rng(7)
    exact = 0
    for (c, A, B), (_, _, dC), r in zip(sample, dev, reps):
        assert r.status == 0 and r.nonfinite == 0 and r.samples >= 64
        assert r.est_err <= TARGET, (c, r.selected, r.slices_used, r.est_err)
        s_cpu, probs = oracle.mlp_select(model, oracle.features(A, B, TARGET), s_cap)
        near = np.any(np.abs(np.cumsum(probs) - model["thr"]) < 1e-5)
        assert r.selected == s_cpu or near, (c, r.selected, s_cpu)
        s = r.slices_used
        assert s == selector.escalation_passes(r.selected, r.repaired, model["fallback"])[-1]
        C = ozg.from_device(dC, c.m, c.n)
        if c.m * c.n * c.k * s * (s + 1) / 2 <= FULL_COMPARE_MACS:
            rows, cols = np.arange(c.m), np.arange(c.n)
        else:
            rows, cols = band_samples(c.m, 128, g), band_samples(c.n, 128, g)
        As, Bs = np.asfortranarray(A[rows]), np.asfortranarray(B[:, cols])
        E = oracle.dgemm_emu(As, Bs, s)
        Cs = C[np.ix_(rows, cols)]
        if windows(s, c.k) <= 2:
            assert np.array_equal(Cs, E), (c, s)
            exact += 1
        else:
            tol = 4 * (s + 2) * U * oracle.abs_product(As, Bs) + 2 * U * np.abs(E)
            assert (np.abs(Cs - E) <= tol).all(), (c, s)
    assert exact >= len(sample) // 2
    ctx.close()


def test_selected_counts_against_oracle_minimal_counts(ozg, sample):
    """Accuracy of the selector's choices on the headline batch: for 32 of the sampled calls the
    oracle labels the minimal count -- the smallest s in 5..13 whose emulation of a 16 x 16 block
    of the product (full k; the same entries as in the full product) is within the target of the
    double-double product, the way the training labels are made -- and the counts the network
    chose in a learned grouped run are compared with it (exact, over, under)."""
    model = selector.read_model(selector.DEFAULT_MODEL)
    sub = sample[::2]
    st = torch.cuda.Stream()
    ctx = ozg.Context(stream=st)
    ctx.load_selector(selector.DEFAULT_MODEL)
    ctx.set_target_error(TARGET)
    ctx.set_check_samples(64)
    dev = [(ozg.to_device(A), ozg.to_device(B), torch.empty((c.n, c.m), dtype=torch.float64, device="cuda"))
           for c, A, B in sub]
    calls = [("N", "N", c.m, c.n, c.k, 1.0, dA, c.m, dB, c.k, 0.0, dC, c.m)
             for (c, _, _), (dA, dB, dC) in zip(sub, dev)]
    with torch.cuda.stream(st):
        reps = ctx.dgemm_grouped(calls, [0] * len(calls), report=True)
    ctx.close()
    g = workloads.rng(11)
    smin = []
    for c, A, B in sub:
        rows = np.sort(g.choice(c.m, min(16, c.m), replace=False))
        cols = np.sort(g.choice(c.n, min(16, c.n), replace=False))
        As, Bs = np.asfortranarray(A[rows]), np.asfortranarray(B[:, cols])
        label = 14
        for s in range(5, 14):
            if oracle.rel_err_vs_dd(oracle.dgemm_emu(As, Bs, s), As, Bs) <= TARGET:
                label = s
                break
        smin.append(label)
    ev = selector.selector_eval([r.selected for r in reps], smin, [c.m * c.n * c.k for c, _, _ in sub])
    assert ev["exact"] >= 0.5 and ev["under"] <= 0.15, ev
    assert ev["mean_selected"] - ev["mean_minimum"] <= 1.0, ev
    assert max(r.selected for r in reps) < model["fallback"]
