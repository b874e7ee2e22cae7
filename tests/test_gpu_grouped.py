"""Grouped emulated DGEMM (one persistent launch over many uneven GEMMs, CUDA-graph replay,
tile-variant autotuner) against the oracle, call by call; the tile variants agree bit for bit."""
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


def make_batch(ozg, count, seed, max_dim=600, beta_zero=False):
    g = workloads.rng(seed)
    batch = []
    for i in range(count):
        m, n, k = (int(x) for x in np.exp(g.uniform(0, np.log(max_dim), 3)).round())
        ta, tb = g.choice(["N", "T"]), g.choice(["N", "T"])
        s = int(g.integers(3, 10))
        alpha = float(g.choice([1.0, -0.5, 2.0]))
        beta = 0.0 if beta_zero else float(g.choice([0.0, 1.0, 0.25]))
        A = workloads.wide_exponent((m, k) if ta == "N" else (k, m), float(g.uniform(0, 3)), g)
        B = workloads.wide_exponent((k, n) if tb == "N" else (n, k), float(g.uniform(0, 3)), g)
        C0 = np.asfortranarray(g.uniform(-1, 1, (m, n)))
        batch.append(dict(ta=ta, tb=tb, m=m, n=n, k=k, s=s, alpha=alpha, beta=beta, A=A, B=B, C0=C0,
                          dA=ozg.to_device(A), dB=ozg.to_device(B), dC=ozg.to_device(C0)))
    return batch


def calls_of(batch):
    return [(b["ta"], b["tb"], b["m"], b["n"], b["k"], b["alpha"], b["dA"], b["A"].shape[0], b["dB"],
             b["B"].shape[0], b["beta"], b["dC"], b["m"]) for b in batch]


def windows(s, k, cplx=False):
    """Exact int64 windows of the default epilogue: the largest group count c with
    (s k_pad 127^2 [x2 complex]) 128^(c-1) 128/127 < 2^63, and ceil(s / c) windows.  k_pad is k
    rounded up to 128 (the 128-wide kernels' padding; the 256-wide ones pad to 64, which never
    needs more windows)."""
    gmax = s * (-(-k // 128) * 128) * 127 * 127 * (2 if cplx else 1)
    c = max(1, (62 - gmax.bit_length()) // 7 + 1)
    return -(-s // c)


def check_batch(ozg, batch):
    """Every call against the oracle's emulation at its count: bit for bit while the epilogue's
    two exact int64 windows cover every group (every call of these batches), else within the
    stated tolerance of the FP64 continuation."""
    for b in batch:
        C = ozg.from_device(b["dC"], b["m"], b["n"])
        E = oracle.dgemm_emu(b["A"], b["B"], b["s"], b["ta"], b["tb"], b["alpha"], b["beta"], b["C0"])
        if windows(b["s"], b["k"]) <= 2:
            assert np.array_equal(C, E), (b["m"], b["n"], b["k"], b["s"])
            continue
        AB = oracle.abs_product(b["A"], b["B"], b["ta"], b["tb"])
        tol = 4 * (b["s"] + 2) * U * abs(b["alpha"]) * AB + 2 * U * np.abs(E) + 2 * U * abs(b["beta"]) * np.abs(b["C0"])
        assert (np.abs(C - E) <= tol).all(), (b["m"], b["n"], b["k"], b["s"])


@pytest.mark.parametrize("graphs", [True, False])
def test_grouped_matches_oracle_and_replays(ozg, graphs):
    st = torch.cuda.Stream()
    ctx = ozg.Context(stream=st)
    ctx.set_graphs(graphs)
    ctx.set_check_samples(16)
    batch = make_batch(ozg, 40, seed=300)
    with torch.cuda.stream(st):
        reps = ctx.dgemm_grouped(calls_of(batch), [b["s"] for b in batch], report=True)
    assert all(r.status == 0 and r.slices_used == b["s"] and r.nonfinite == 0 for r, b in zip(reps, batch))
    assert all(0 <= r.est_err < 1e-3 for r in reps)
    check_batch(ozg, batch)
    # replay (graph) with new contents in the same buffers
    g = workloads.rng(301)
    for b in batch:
        b["A"] = np.asfortranarray(b["A"] * g.uniform(0.5, 2.0))
        b["dA"].copy_(ozg.to_device(b["A"]))
        b["C0"] = np.asfortranarray(g.uniform(-1, 1, (b["m"], b["n"])))
        b["dC"].copy_(ozg.to_device(b["C0"]))
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        ctx.dgemm_grouped(calls_of(batch), [b["s"] for b in batch])
    ctx.sync()
    check_batch(ozg, batch)
    ctx.close()


def test_grouped_autotune_bit_identical_and_nonfinite(ozg, tmp_path):
    st = torch.cuda.Stream()
    batch = make_batch(ozg, 24, seed=310, beta_zero=True)
    batch[5]["A"][0, 0] = np.nan
    batch[5]["dA"].copy_(ozg.to_device(batch[5]["A"]))
    outs = []
    for tune in (False, True):
        ctx = ozg.Context(stream=st)
        ctx.set_autotune(tune, str(tmp_path / "tune.txt"))
        for b in batch:
            b["dC"].zero_()
        torch.cuda.synchronize()
        with torch.cuda.stream(st):
            reps = ctx.dgemm_grouped(calls_of(batch), [b["s"] for b in batch], report=True)
        assert reps[5].nonfinite == 1 and reps[5].slices_used == -1
        outs.append([b["dC"].clone() for b in batch])
        ctx.close()
    for x, y in zip(*outs):
        assert torch.equal(torch.nan_to_num(x, nan=7.0), torch.nan_to_num(y, nan=7.0))
    b = batch[5]
    C = ozg.from_device(b["dC"], b["m"], b["n"])
    ref = oracle.dgemm_naive(b["A"], b["B"], b["ta"], b["tb"], b["alpha"])
    assert np.array_equal(np.isnan(C), np.isnan(ref))
    others = [x for i, x in enumerate(batch) if i != 5]
    check_batch(ozg, others)


def test_grouped_edge_calls_and_invalid(ozg):
    ctx = ozg.Context()
    A, B = workloads.uniform_pair(20, 10, 30, seed=320)
    dA, dB = ozg.to_device(A), ozg.to_device(B)
    C0 = np.asfortranarray(workloads.rng(321).uniform(-1, 1, (20, 10)))
    dC1, dC2, dC3 = ozg.to_device(C0), ozg.to_device(C0), ozg.to_device(C0)
    calls = [("N", "N", 20, 10, 30, 1.0, dA, 20, dB, 30, 0.0, dC1, 20),
             ("N", "N", 20, 10, 0, 1.0, dA, 20, dB, 30, 2.0, dC2, 20),    # k == 0: C = beta C
             ("N", "N", 20, 10, 30, 0.0, dA, 20, dB, 30, 0.5, dC3, 20)]   # alpha == 0
    ctx.dgemm_grouped(calls, [7, 7, 7])
    ctx.sync()
    assert np.array_equal(ozg.from_device(dC1, 20, 10), oracle.dgemm_emu(A, B, 7))
    assert np.array_equal(ozg.from_device(dC2, 20, 10), 2.0 * C0)
    assert np.array_equal(ozg.from_device(dC3, 20, 10), 0.5 * C0)
    bad = [("N", "N", 20, 10, 30, 1.0, dA, 19, dB, 30, 0.0, dC1, 20)]
    with pytest.raises(ozg.OzgError):
        ctx.dgemm_grouped(bad, [7])
    ctx.close()


def test_single_call_autotune_cache_and_bits(ozg, tmp_path):
    m, n, k, s = 300, 200, 500, 6
    A, B = workloads.wide_exponent_pair(m, n, k, 1.0, seed=330)
    dA, dB = ozg.to_device(A), ozg.to_device(B)
    res = []
    path = tmp_path / "single.txt"
    for tune in (False, True, True):
        ctx = ozg.Context()
        ctx.set_autotune(tune, str(path))
        dC = torch.zeros((n, m), dtype=torch.float64, device="cuda")
        ctx.dgemm("N", "N", m, n, k, 1.0, dA, m, dB, k, 0.0, dC, m, s)
        ctx.sync()
        res.append(dC.clone())
        ctx.close()
    assert torch.equal(res[0], res[1]) and torch.equal(res[1], res[2])
    lines = path.read_text().split()
    assert len(lines) == 2 and lines[1] in ("0", "1", "2", "3", "5")  # one bucket tuned once, then read back


def test_tile_variants_bit_identical(ozg):
    """The tile variants (128 x 256 / 128 x 128 tiles, immediate / deferred epilogue pushes, CTA
    pairs on 256 x 128 tiles, and group pairs stacked into N = 256 MMAs) give the same bits: single real and complex calls with
    beta != 0, and a grouped batch."""
    m, n, k, s = 200, 300, 2100, 8   # ragged tiles, several k-segments per pair
    A, B = workloads.wide_exponent_pair(m, n, k, 1.0, seed=340)
    C0 = np.asfortranarray(workloads.rng(341).uniform(-1, 1, (m, n)))
    Z = workloads.kkr_like_pair(nblk=5, bs=32, seed=342)
    mz, nz, kz = 150, 97, 160
    Az, Bz = np.asfortranarray(Z[0][:mz, :kz]), np.asfortranarray(Z[1][:kz, :nz])
    Z0 = np.asfortranarray(workloads.rng(343).normal(size=(mz, nz)) + 1j * workloads.rng(344).normal(size=(mz, nz)))
    batch = make_batch(ozg, 12, seed=345)
    dA, dB, dAz, dBz = (ozg.to_device(x) for x in (A, B, Az, Bz))
    res = []
    for v in range(6):  # variant 4 (CTA pairs) runs the grouped batch on 2-CTA clusters
        ctx = ozg.Context()
        ctx.set_tile_variant(v)
        dC, dZ = ozg.to_device(C0), ozg.to_device(Z0)
        ctx.dgemm("N", "N", m, n, k, -0.5, dA, m, dB, k, 0.75, dC, m, s)
        ctx.zgemm("N", "N", mz, nz, kz, 0.5 - 2j, dAz, mz, dBz, kz, 1.5 + 0.25j, dZ, mz, 6)
        for b in batch:
            b["dC"].copy_(ozg.to_device(b["C0"]))
        torch.cuda.synchronize()
        ctx.dgemm_grouped(calls_of(batch), [b["s"] for b in batch])
        ctx.sync()
        res.append([dC.clone(), dZ.clone()] + [b["dC"].clone() for b in batch])
        ctx.close()
    for r in res[1:]:
        assert all(torch.equal(x, y) for x, y in zip(res[0], r))
    check_batch(ozg, batch)
    assert windows(s, k) <= 2
    E = oracle.dgemm_emu(A, B, s, "N", "N", -0.5, 0.75, C0)
    assert np.array_equal(ozg.from_device(res[0][0], m, n), E)
    Ez = oracle.zgemm_emu(Az, Bz, 6, "N", "N", 0.5 - 2j, 1.5 + 0.25j, Z0)
    assert np.array_equal(ozg.from_device(res[0][1], mz, nz), Ez)
    with pytest.raises(ozg.OzgError):
        ozg.Context().set_tile_variant(6)


NARROW_SHAPES = [(130, 1, 17), (33, 17, 1), (97, 40, 70), (1, 65, 33), (130, 161, 130), (65, 304, 47),
                 (200, 100, 1000), (129, 48, 16)]


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5])
def test_narrow_tiles_ragged_k_bit_exact(ozg, variant):
    """Narrow last column tiles (1 .. 48 valid columns of a 128- or 256-wide tile), k ending
    inside a 16-wide step or a 64-wide TMA box, and row tiles with one to a few valid rows: in
    every tile variant, single real and complex calls and a grouped batch of the same shapes
    equal the oracle bit for bit (s = 7 uses at most two exact windows at any k)."""
    s = 7
    ctx = ozg.Context()
    ctx.set_tile_variant(variant)
    try:
        batch = []
        for i, (m, n, k) in enumerate(NARROW_SHAPES):
            g = workloads.rng(900 + i)
            A = np.asfortranarray(workloads.wide_exponent((m, k), 2.0, g))
            B = np.asfortranarray(workloads.wide_exponent((k, n), 2.0, g))
            C0 = np.asfortranarray(g.uniform(-1, 1, (m, n)))
            dC = ozg.to_device(C0)
            ctx.dgemm("N", "N", m, n, k, -0.5, ozg.to_device(A), m, ozg.to_device(B), k, 0.75, dC, m, s)
            ctx.sync()
            E = oracle.dgemm_emu(A, B, s, "N", "N", -0.5, 0.75, C0)
            assert np.array_equal(ozg.from_device(dC, m, n), E), (m, n, k)
            batch.append(dict(ta="N", tb="N", m=m, n=n, k=k, s=s, alpha=-0.5, beta=0.75, A=A, B=B, C0=C0,
                              dA=ozg.to_device(A), dB=ozg.to_device(B), dC=ozg.to_device(C0)))
        ctx.dgemm_grouped(calls_of(batch), [s] * len(batch))
        ctx.sync()
        for b in batch:
            E = oracle.dgemm_emu(b["A"], b["B"], s, "N", "N", -0.5, 0.75, b["C0"])
            assert np.array_equal(ozg.from_device(b["dC"], b["m"], b["n"]), E), (b["m"], b["n"], b["k"])
        for i, (m, n, k) in enumerate([(45, 9, 23), (130, 70, 50), (3, 130, 17)]):
            g = workloads.rng(950 + i)
            A = np.asfortranarray(workloads.wide_exponent((m, k), 1.0, g) + 1j * workloads.wide_exponent((m, k), 1.0, g))
            B = np.asfortranarray(workloads.wide_exponent((k, n), 1.0, g) + 1j * workloads.wide_exponent((k, n), 1.0, g))
            C0 = np.asfortranarray(g.normal(size=(m, n)) + 1j * g.normal(size=(m, n)))
            dC = ozg.to_device(C0)
            ctx.zgemm("N", "T" if i == 1 else "N", m, n, k, 0.5 - 2j, ozg.to_device(A), m,
                      ozg.to_device(np.asfortranarray(B.T) if i == 1 else B), n if i == 1 else k, 1.5 + 0.25j, dC, m, s)
            ctx.sync()
            E = oracle.zgemm_emu(A, np.asfortranarray(B.T) if i == 1 else B, s, "N", "T" if i == 1 else "N",
                                 0.5 - 2j, 1.5 + 0.25j, C0)
            assert np.array_equal(ozg.from_device(dC, m, n), E), (m, n, k)
    finally:
        ctx.close()


@pytest.mark.parametrize("s", [1, 2, 3, 5, 8, 10, 11, 13, 16, 17])
def test_stacked_group_pairs_match_one_group_kernel(ozg, s):
    """Stacked group pairs (variant 5): windows with an odd group count (a lone first group),
    one to three windows, k sweeps over several chains and ragged k; single real and complex
    calls with alpha / beta and a grouped batch give the bits of the one-group 128-wide kernel
    (variant 1), and the oracle's where the exact sum needs at most two windows.  s = 17 is above
    the stacked kernel's limit and runs as variant 1."""
    # k mod 64 covers every count of valid 16-wide slices in the last k sub-tile (k16 = 4, 3, 4,
    # 1, 2, 1), and k = 7 is one sub-tile that is both the first and the last of every sweep
    shapes = [(200, 130, 2100), (129, 257, 1000), (64, 64, 64), (130, 70, 129), (97, 33, 85), (40, 150, 7)]
    res = {}
    for v in (1, 5):
        ctx = ozg.Context()
        ctx.set_tile_variant(v)
        try:
            out = []
            batch = []
            for i, (m, n, k) in enumerate(shapes):
                g = workloads.rng(1500 + i)
                A = np.asfortranarray(workloads.wide_exponent((m, k), 1.5, g))
                B = np.asfortranarray(workloads.wide_exponent((k, n), 1.5, g))
                C0 = np.asfortranarray(g.uniform(-1, 1, (m, n)))
                dC = ozg.to_device(C0)
                ctx.dgemm("N", "N", m, n, k, -0.5, ozg.to_device(A), m, ozg.to_device(B), k, 0.75, dC, m, s)
                ctx.sync()
                out.append(ozg.from_device(dC, m, n))
                if windows(s, k) <= 2:
                    assert np.array_equal(out[-1], oracle.dgemm_emu(A, B, s, "N", "N", -0.5, 0.75, C0)), (m, n, k)
                batch.append(dict(ta="N", tb="N", m=m, n=n, k=k, s=s, alpha=1.0, beta=0.0, A=A, B=B, C0=C0,
                                  dA=ozg.to_device(A), dB=ozg.to_device(B), dC=ozg.to_device(C0)))
            ctx.dgemm_grouped(calls_of(batch), [s] * len(batch))
            ctx.sync()
            for b in batch:
                out.append(ozg.from_device(b["dC"], b["m"], b["n"]))
                if windows(s, b["k"]) <= 2:
                    assert np.array_equal(out[-1], oracle.dgemm_emu(b["A"], b["B"], s)), (b["m"], b["n"], b["k"])
            m, n, k = 45, 70, 333
            g = workloads.rng(1600)
            A = np.asfortranarray(workloads.wide_exponent((m, k), 1.0, g) + 1j * workloads.wide_exponent((m, k), 1.0, g))
            B = np.asfortranarray(workloads.wide_exponent((k, n), 1.0, g) + 1j * workloads.wide_exponent((k, n), 1.0, g))
            C0 = np.asfortranarray(g.normal(size=(m, n)) + 1j * g.normal(size=(m, n)))
            dC = ozg.to_device(C0)
            ctx.zgemm("N", "N", m, n, k, 0.5 - 2j, ozg.to_device(A), m, ozg.to_device(B), k, 1.5 + 0.25j, dC, m, s)
            ctx.sync()
            out.append(ozg.from_device(dC, m, n))
            if windows(s, k, cplx=True) <= 2:
                assert np.array_equal(out[-1], oracle.zgemm_emu(A, B, s, "N", "N", 0.5 - 2j, 1.5 + 0.25j, C0))
            res[v] = out
        finally:
            ctx.close()
    for x, y in zip(res[1], res[5]):
        assert np.array_equal(x, y)


def test_pair_tiles_bit_exact_and_replay(ozg):
    """CTA pairs (variant 4): a batch whose calls give pair tiles with both halves full, a ragged
    second half, an all-padding second half (m <= 128), one column and many pair tiles, with
    alpha / beta, a call skipped for a NaN, fewer CTAs than pair tiles (the persistent loop) and a
    graph replay; every finite call equals the oracle bit for bit."""
    shapes = [(256, 128, 300), (300, 129, 64), (100, 250, 1000), (513, 1, 17), (700, 900, 129), (128, 128, 2100),
              (257, 384, 640), (1200, 1100, 333)]
    st = torch.cuda.Stream()
    ctx = ozg.Context(stream=st)
    ctx.set_tile_variant(4)
    batch = []
    for i, (m, n, k) in enumerate(shapes):
        g = workloads.rng(1300 + i)
        A = np.asfortranarray(workloads.wide_exponent((m, k), 2.0, g))
        B = np.asfortranarray(workloads.wide_exponent((k, n), 2.0, g))
        C0 = np.asfortranarray(g.uniform(-1, 1, (m, n)))
        alpha, beta = (1.0, 0.0) if i % 2 == 0 else (-0.5, 0.75)
        batch.append(dict(ta="N", tb="N", m=m, n=n, k=k, s=7 + i % 3, alpha=alpha, beta=beta, A=A, B=B, C0=C0,
                          dA=ozg.to_device(A), dB=ozg.to_device(B), dC=ozg.to_device(C0)))
    bad = batch[3]
    bad["A"][5, 0] = np.nan
    bad["dA"].copy_(ozg.to_device(bad["A"]))
    torch.cuda.synchronize()
    for rep in range(2):  # plan + capture, then a replay with the same buffers
        for b in batch:
            b["dC"].copy_(ozg.to_device(b["C0"]))
        torch.cuda.synchronize()
        with torch.cuda.stream(st):
            reps = ctx.dgemm_grouped(calls_of(batch), [b["s"] for b in batch], report=True)
        assert reps[3].nonfinite == 1
        assert all(r.status == 0 for r in reps)
        check_batch(ozg, [b for i, b in enumerate(batch) if i != 3])
    ctx.close()
