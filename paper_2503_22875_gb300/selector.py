"""Learned slice selector: model files, training data and training (the adaptive split number
proposed in Sec. 4 of the paper: choose, per GEMM, the smallest split number that meets the
accuracy it needs).

* Features come from the library's own feature kernels (``ozg_selector_features``).
* Labels: for each training GEMM, the library emulates a block of 16 sampled rows x 16 sampled
  columns (full k) at every s in 2..12 in grouped launches, and its GPU double-double check
  measures the componentwise error; the label is the smallest s whose error meets the target
  (s = 12 if none does).  Per-row and per-column scales make the block's emulation identical to
  the full product's on those entries.
* Training runs on the GPU with the library's forward/backward and Adam kernels
  (``ozg_selector_train_step``) on four fifths of the GEMMs.
* Decision: the smallest s whose cumulative predicted probability of "s_min <= s" reaches a
  threshold, chosen on the held-out fifth to minimise the expected tensor work -- s(s+1)/2
  products at the chosen s plus a re-run at the fallback count when the sampled check rejects
  the result (s below the GEMM's minimal sufficient count).

    python -m paper_2503_22875_gb300.selector --problems 25000 --out model.ozgsel
"""
from __future__ import annotations

import argparse
import json
import os
import struct
import time

import numpy as np

S_LO = 2
N_CLASSES = 11
N_IN, N_H = 24, 64
PARAMS = N_H * N_IN + N_H + N_H * N_H + N_H + N_CLASSES * N_H + N_CLASSES
TARGETS = (1e-10, 1e-14)
DATA_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
# the model the benchmark and the headline tests load
DEFAULT_MODEL = os.path.join(DATA_DIR, "selector_v1.ozgsel")
S_MEASURE = 16  # errors are measured up to s = 16; classes stop at s = 12


# ------------------------------------------------------------------------------------ model files
def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 values to BF16 (nearest, ties to even) and return the 16-bit patterns."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (u & 0xFFFF).astype(np.uint16)


def split_theta(theta: np.ndarray):
    t = np.asarray(theta, dtype=np.float32)
    o = 0
    parts = {}
    for name, size in (("W1", N_H * N_IN), ("b1", N_H), ("W2", N_H * N_H), ("b2", N_H), ("W3", N_CLASSES * N_H),
                       ("b3", N_CLASSES)):
        parts[name] = t[o:o + size]
        o += size
    return parts


def write_model(path: str, theta, mean, std, thr: float, fallback: int, s_lo: int = S_LO) -> None:
    p = split_theta(theta)
    with open(path, "wb") as f:
        f.write(b"OZGSEL01")
        f.write(struct.pack("<6i", 1, N_IN, N_H, N_CLASSES, s_lo, fallback))
        f.write(struct.pack("<f", thr))
        f.write(np.asarray(mean, "<f4").tobytes())
        f.write(np.asarray(std, "<f4").tobytes())
        for w, b in (("W1", "b1"), ("W2", "b2"), ("W3", "b3")):
            f.write(to_bf16_bits(p[w]).astype("<u2").tobytes())
            f.write(np.asarray(p[b], "<f4").tobytes())


def read_model(path: str) -> dict:
    with open(path, "rb") as f:
        data = f.read()
    assert data[:8] == b"OZGSEL01"
    ver, nin, nh, nout, s_lo, fallback = struct.unpack("<6i", data[8:32])
    thr = struct.unpack("<f", data[32:36])[0]
    o = 36

    def take(dt, n):
        nonlocal o
        a = np.frombuffer(data, dtype=dt, count=n, offset=o).copy()
        o += a.nbytes
        return a

    mean = take("<f4", nin)
    std = take("<f4", nin)
    m = dict(mean=mean, std=std, inv_std=np.where(std > 0, np.float32(1) / std, np.float32(0)).astype(np.float32),
             thr=thr, s_lo=s_lo, fallback=fallback)
    m["W1"], m["b1"] = take("<u2", nh * nin), take("<f4", nh)
    m["W2"], m["b2"] = take("<u2", nh * nh), take("<f4", nh)
    m["W3"], m["b3"] = take("<u2", nout * nh), take("<f4", nout)
    return m


# ------------------------------------------------------------------------------------ data
def make_dataset(ctx, problems: int, seed: int = 5, lo: int = 64, hi: int = 4096, phi_hi: float = 6.0,
                 block: int = 16, samples: int = 256, chunk: int = 256, targets=TARGETS, log=None,
                 keep_blocks: bool = False):
    """(X, y, meta): features (float32 [len(targets) * problems, 24]), labels (class = s - 2) and
    the problem shapes.  ctx is an ozg.Context; all GPU work goes through the library."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    dims = np.exp(rng.uniform(np.log(lo), np.log(hi), size=(problems, 3))).round().astype(int)
    phis = rng.uniform(0.0, phi_hi, size=problems)
    feats = np.zeros((problems, N_IN), np.float32)
    n_meas = S_MEASURE - S_LO + 1
    errs = np.zeros((problems, n_meas))
    feat_dev = torch.empty(N_IN, dtype=torch.float32, device="cuda")
    kept = []
    ctx.set_check_samples(samples)
    t0 = time.time()
    for c0 in range(0, problems, chunk):
        c1 = min(problems, c0 + chunk)
        blocks = []
        for p in range(c0, c1):
            m, n, k = (int(x) for x in dims[p])
            phi = float(phis[p])

            def draw(rows, cols):  # column-major rows x cols as a (cols, rows) tensor
                u = torch.rand((cols, rows), generator=gen, device="cuda", dtype=torch.float64)
                z = torch.randn((cols, rows), generator=gen, device="cuda", dtype=torch.float64)
                return (u - 0.5) * torch.exp(phi * z)

            A, B = draw(m, k), draw(k, n)
            ctx.selector_features("N", "N", m, n, k, A, m, B, k, feat_dev)
            feats[p] = feat_dev.cpu().numpy()
            ri = torch.from_numpy(rng.choice(m, size=min(block, m), replace=False)).cuda()
            ci = torch.from_numpy(rng.choice(n, size=min(block, n), replace=False)).cuda()
            blocks.append((A[:, ri].contiguous(), B[ci, :].contiguous(), k))
        calls, slices, outs = [], [], []
        for (As, Bs, k) in blocks:
            bm, bn = As.shape[1], Bs.shape[0]
            # As: (k, bm) column-major bm x k; Bs: (bn, k) holds column-major k x bn
            for s in range(S_LO, S_MEASURE + 1):
                C = torch.empty((bn, bm), dtype=torch.float64, device="cuda")
                calls.append(("N", "N", bm, bn, k, 1.0, As, bm, Bs, k, 0.0, C, bm))
                slices.append(s)
                outs.append(C)
        reps = ctx.dgemm_grouped(calls, slices, report=True)
        if keep_blocks:
            kept.extend((As.cpu().numpy(), Bs.cpu().numpy()) for As, Bs, _ in blocks)
        e = np.array([r.est_err for r in reps]).reshape(c1 - c0, n_meas)
        errs[c0:c1] = e
        if log:
            log(f"  {c1}/{problems} problems, {time.time() - t0:.1f} s")
    X, y, smin = [], [], []
    for t in targets:
        ft = feats.copy()
        ft[:, 23] = np.float32(np.log10(t))
        ok = errs <= t
        first = np.where(ok.any(1), ok.argmax(1), n_meas)  # index of the minimal sufficient s
        X.append(ft)
        y.append(np.minimum(first, N_CLASSES - 1).astype(np.int32))
        smin.append(S_LO + first)  # S_MEASURE + 1 means "more than measured"
    meta = {"dims": dims, "phis": phis, "errs": errs, "blocks": kept, "s_min": np.concatenate(smin)}
    return np.concatenate(X), np.concatenate(y), meta


# ------------------------------------------------------------------------------------ training
def init_params(seed: int) -> np.ndarray:
    r = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for fan_out, fan_in in ((N_H, N_IN), (N_H, N_H), (N_CLASSES, N_H)):
        parts.append(r.normal(0, np.sqrt(2.0 / fan_in), fan_out * fan_in).astype(np.float32))
        parts.append(np.zeros(fan_out, np.float32))
    return np.concatenate(parts)


def train(ctx, X: np.ndarray, y: np.ndarray, epochs: int = 40, batch: int = 1024, lr: float = 2e-3, seed: int = 0,
          log=None):
    """Train on the GPU; returns (theta, mean, std, losses)."""
    import torch
    mean = X.mean(0).astype(np.float32)
    std = (X.std(0) + 1e-6).astype(np.float32)
    std[23] = max(std[23], 1.0)
    Xn = ((X - mean) / std).astype(np.float32)
    dX = torch.from_numpy(Xn).cuda()
    dy = torch.from_numpy(y.astype(np.int32)).cuda()
    ctx.selector_set_params(init_params(seed))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    n = len(y)
    losses = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen, device="cuda")
        Xp, yp = dX[perm].contiguous(), dy[perm].contiguous()
        tot = 0.0
        for b0 in range(0, n, batch):
            B = min(batch, n - b0)
            tot += ctx.selector_train_step(Xp[b0:b0 + B], yp[b0:b0 + B], B, lr) * B
        losses.append(tot / n)
        if log and (ep % 10 == 0 or ep == epochs - 1):
            log(f"  epoch {ep}: loss {losses[-1]:.4f}")
    return ctx.selector_get_params(), mean, std, losses


def predict_probs(theta, mean, std, X: np.ndarray) -> np.ndarray:
    """Class probabilities of the model as the GPU computes them (BF16 weights, FP32 arithmetic;
    the summation order may differ in the last bits)."""
    p = split_theta(theta)
    inv = np.where(std > 0, np.float32(1) / np.asarray(std, np.float32), np.float32(0)).astype(np.float32)

    def bf(w, shape):
        return (to_bf16_bits(w).astype(np.uint32) << 16).view(np.float32).reshape(shape)
    x = ((np.asarray(X, np.float32) - np.asarray(mean, np.float32)) * inv).astype(np.float32)
    h1 = np.maximum(x @ bf(p["W1"], (N_H, N_IN)).T + p["b1"], 0).astype(np.float32)
    h2 = np.maximum(h1 @ bf(p["W2"], (N_H, N_H)).T + p["b2"], 0).astype(np.float32)
    z = (h2 @ bf(p["W3"], (N_CLASSES, N_H)).T + p["b3"]).astype(np.float32)
    z -= z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def decide(probs: np.ndarray, thr: float, fallback: int, s_lo: int = S_LO) -> np.ndarray:
    """The decision rule: the smallest s whose cumulative probability of 's_min <= s' reaches thr."""
    cum = np.cumsum(probs, axis=1)
    hit = cum >= thr
    return np.where(hit.any(1), s_lo + hit.argmax(1), fallback)


def choose_threshold(probs, s_min, work, fallback, grid=None):
    """Threshold minimising the expected tensor work on held-out GEMMs: s(s+1)/2 products at the
    chosen s, plus a re-run at the fallback count whenever s is below the GEMM's minimal
    sufficient count (the sampled check rejects it).  work: m n k per sample."""
    grid = grid if grid is not None else [0.5, 0.6, 0.7, 0.8, 0.85, 0.9, 0.93, 0.95, 0.97, 0.98, 0.99, 0.995]
    fb_cost = fallback * (fallback + 1) / 2
    table = {}
    for thr in grid:
        s = decide(probs, thr, fallback)
        miss = s < s_min
        cost = float(np.sum(work * (s * (s + 1) / 2 + miss * fb_cost)))
        table[thr] = {"cost": cost, "rerun_frac": float(miss.mean()), "mean_s": float(s.mean())}
    best = min(table, key=lambda t: table[t]["cost"])
    return best, table


def fallback_from_smin(s_min: np.ndarray, q: float = 99.9) -> int:
    """The conservative fixed count: the q-th percentile of the training GEMMs' minimal
    sufficient slice counts (measured up to s = 16), capped to the library's maximum of 18."""
    return int(min(18, np.percentile(s_min, q, method="higher")))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", type=int, default=25000)
    ap.add_argument("--lo", type=int, default=64)
    ap.add_argument("--hi", type=int, default=4096)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--threshold", type=float, default=0.0,
                    help="decision threshold; <= 0 chooses it on held-out GEMMs by expected work")
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--out", required=True)
    args = ap.parse_args()
    from . import build, ozg
    build.build()
    ctx = ozg.Context()
    t0 = time.time()
    X, y, meta = make_dataset(ctx, args.problems, seed=args.seed, lo=args.lo, hi=args.hi, log=print)
    t1 = time.time()
    # every fifth GEMM is held out to choose the decision threshold
    prob_idx = np.arange(len(y)) % args.problems
    held = prob_idx % 5 == 0
    theta, mean, std, losses = train(ctx, X[~held], y[~held], epochs=args.epochs, log=print)
    t2 = time.time()
    fb = fallback_from_smin(meta["s_min"])
    thr = args.threshold
    table = None
    if thr <= 0:
        dims = meta["dims"][prob_idx[held]]
        work = dims[:, 0].astype(float) * dims[:, 1] * dims[:, 2]
        thr, table = choose_threshold(predict_probs(theta, mean, std, X[held]), meta["s_min"][held], work, fb)
    write_model(args.out, theta, mean, std, thr, fb)
    print(json.dumps({"problems": args.problems, "samples": int(len(y)), "held_out": int(held.sum()),
                      "data_s": t1 - t0, "train_s": t2 - t1, "final_loss": losses[-1], "first_loss": losses[0],
                      "fallback": fb, "threshold": thr, "threshold_table": table,
                      "label_hist": np.bincount(y, minlength=N_CLASSES).tolist(),
                      "s_min_hist": np.bincount(meta["s_min"], minlength=S_MEASURE + 2).tolist()}))


if __name__ == "__main__":
    main()
