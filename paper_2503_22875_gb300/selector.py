"""Learned slice selector: model files, training data and training (the adaptive split number
proposed in Sec. 4 of the paper: choose, per GEMM, the smallest split number that meets the
accuracy it needs).

* Features come from the library's own feature kernels (``ozg_selector_features``).
* Labels: for each training GEMM, the library emulates a block of 16 sampled rows x 16 sampled
  columns (full k) at every s in 2..16 in grouped launches, and its GPU double-double check
  measures the componentwise error; the label is the smallest s whose error meets the target
  (class 12 if none up to 12 does).  Per-row and per-column scales make the block's emulation
  identical to the full product's on those entries.  Labels are made for every decade of target
  from 1e-10 to 1e-14 from the same error measurements: the target is an input of the network,
  and with labels at 1e-10 and 1e-14 only it interpolates poorly in between (on the grouped
  batch's distribution at 1e-12, the most likely class was the minimal count for 28% of the
  GEMMs, against 87% with labels at every decade).
* Training runs on the GPU with the library's forward/backward and Adam kernels
  (``ozg_selector_train_step``).
* Decision: the smallest s whose cumulative predicted probability of "s_min <= s" reaches a
  threshold.  The threshold minimises the expected tensor work on a calibration set drawn from
  the workload the model serves (by default the grouped batch's distribution: sizes 32..2048,
  phi ~ U(0, 4), target 1e-12; other seeds than any benchmark batch): s(s+1)/2 products at the
  chosen s, plus the escalation the sampled check triggers when s is below the GEMM's minimal
  sufficient count -- a re-run at min(s + 2, fallback) and, if that is still short, one at the
  fallback.  Without a calibration set, a held-out fifth of the training GEMMs serves.

    python -m paper_2503_22875_gb300.selector --problems 50000 --out model.ozgsel
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
TARGETS = (1e-10, 1e-11, 1e-12, 1e-13, 1e-14)
ESCALATION_STEP = 2  # a rejected count s is re-run at min(s + 2, fallback), then at the fallback
DATA_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
# the model the benchmark and the headline tests load
DEFAULT_MODEL = os.path.join(DATA_DIR, "selector_v3.ozgsel")
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


def escalation_work(s1, s_min, fallback, step=ESCALATION_STEP):
    """Slice products (s(s+1)/2 per pass, per unit of m n k) of the check-driven policy for each
    GEMM: the pass at s1; when s1 < s_min (the check rejects it) a pass at s2 = min(s1 + step,
    fallback); when s2 < s_min too and s2 < fallback, a pass at the fallback.  Counts at or above
    the fallback are not escalated.  Returns (products, passes) per GEMM."""
    s1 = np.asarray(s1)
    s_min = np.asarray(s_min)
    s2 = np.minimum(s1 + step, fallback)
    miss1 = (s1 < s_min) & (s1 < fallback)
    miss2 = miss1 & (s2 < s_min) & (s2 < fallback)
    prod = s1 * (s1 + 1) / 2 + miss1 * s2 * (s2 + 1) / 2 + miss2 * fallback * (fallback + 1) / 2
    return prod, 1 + miss1.astype(int) + miss2.astype(int)


def escalation_passes(selected: int, repaired: int, fallback: int, step: int = ESCALATION_STEP):
    """Slice counts of the passes a learned call of a grouped launch ran, from its report: the
    selected count, then min(selected + step, fallback) for a first re-run and the fallback for a
    second one."""
    seq = [selected]
    if repaired >= 1:
        seq.append(min(selected + step, fallback))
    if repaired >= 2:
        seq.append(fallback)
    return seq


def write_constant_model(path: str, s: int, fallback: int) -> None:
    """A model file whose decision is always s (zero weights, a one-hot last bias; the class range
    is shifted up when s is above 12): a fixed count run through the learned pipeline -- the same
    feature pass, check and escalation -- to measure what the network's choice gains."""
    theta = np.zeros(PARAMS, dtype=np.float32)
    theta[PARAMS - N_CLASSES:] = -30.0
    s_lo = max(S_LO, s - (N_CLASSES - 1))
    theta[PARAMS - N_CLASSES + (s - s_lo)] = 30.0
    write_model(path, theta, np.zeros(N_IN, np.float32), np.ones(N_IN, np.float32), 0.5, fallback, s_lo=s_lo)


def choose_threshold(probs, s_min, work, fallback, grid=None):
    """Threshold minimising the expected tensor work on calibration GEMMs under the
    check-driven escalation (escalation_work).  work: m n k per sample."""
    grid = grid if grid is not None else [0.5, 0.6, 0.7, 0.8, 0.85, 0.9, 0.93, 0.95, 0.97, 0.98, 0.99, 0.995]
    table = {}
    for thr in grid:
        s = decide(probs, thr, fallback)
        prod, passes = escalation_work(s, s_min, fallback)
        table[thr] = {"cost": float(np.sum(work * prod)), "rerun_frac": float(np.mean(passes > 1)),
                      "second_rerun_frac": float(np.mean(passes > 2)), "mean_s": float(s.mean())}
    best = min(table, key=lambda t: table[t]["cost"])
    return best, table


def selector_eval(selected, s_min, work=None):
    """Accuracy of chosen slice counts against the minimal sufficient counts: the shares of GEMMs
    whose choice is exact, above (over) or below (under) the minimum, the mean number of slices
    above the minimum over the GEMMs that are over, the mean shortfall over those under, and,
    with work (m n k per GEMM), the work-weighted shares."""
    sel = np.asarray(selected, dtype=float)
    smin = np.asarray(s_min, dtype=float)
    d = sel - smin
    out = {"calls": int(len(sel)), "exact": float(np.mean(d == 0)), "over": float(np.mean(d > 0)),
           "under": float(np.mean(d < 0)),
           "mean_excess_slices_when_over": float(d[d > 0].mean()) if np.any(d > 0) else 0.0,
           "mean_shortfall_when_under": float(-d[d < 0].mean()) if np.any(d < 0) else 0.0,
           "mean_selected": float(sel.mean()), "mean_minimum": float(smin.mean())}
    if work is not None:
        w = np.asarray(work, dtype=float)
        out["work_weighted"] = {"exact": float(w[d == 0].sum() / w.sum()), "over": float(w[d > 0].sum() / w.sum()),
                                "under": float(w[d < 0].sum() / w.sum())}
    return out


def fallback_from_smin(s_min: np.ndarray, q: float = 99.9) -> int:
    """The conservative fixed count: the q-th percentile of the training GEMMs' minimal
    sufficient slice counts (measured up to s = 16), capped to the library's maximum of 18."""
    return int(min(18, np.percentile(s_min, q, method="higher")))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", type=int, default=50000)
    ap.add_argument("--lo", type=int, default=32)
    ap.add_argument("--hi", type=int, default=4096)
    ap.add_argument("--phi-hi", type=float, default=6.0)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--threshold", type=float, default=0.0,
                    help="decision threshold; <= 0 chooses it by expected work on the calibration set")
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--cal-problems", type=int, default=12000,
                    help="calibration GEMMs for the threshold (0: a held-out fifth of the training GEMMs)")
    ap.add_argument("--cal-lo", type=int, default=32)
    ap.add_argument("--cal-hi", type=int, default=2048)
    ap.add_argument("--cal-phi-hi", type=float, default=4.0)
    ap.add_argument("--cal-target", type=float, default=1e-12)
    ap.add_argument("--cal-seed", type=int, default=11)
    ap.add_argument("--out", required=True)
    ap.add_argument("--record", default="", help="write the training record (JSON) here")
    args = ap.parse_args()
    from . import build, ozg
    build.build()
    ctx = ozg.Context()
    t0 = time.time()
    X, y, meta = make_dataset(ctx, args.problems, seed=args.seed, lo=args.lo, hi=args.hi, phi_hi=args.phi_hi,
                              log=print)
    prob_idx = np.arange(len(y)) % args.problems
    if args.cal_problems > 0:
        Xc, _, mc = make_dataset(ctx, args.cal_problems, seed=args.cal_seed, lo=args.cal_lo, hi=args.cal_hi,
                                 phi_hi=args.cal_phi_hi, targets=(args.cal_target,), log=print)
        train_mask = np.ones(len(y), dtype=bool)
        cal_smin, cal_dims = mc["s_min"], mc["dims"]
    else:  # every fifth training GEMM is held out
        train_mask = prob_idx % 5 != 0
        Xc, cal_smin, cal_dims = X[~train_mask], meta["s_min"][~train_mask], meta["dims"][prob_idx[~train_mask]]
    t1 = time.time()
    theta, mean, std, losses = train(ctx, X[train_mask], y[train_mask], epochs=args.epochs, log=print)
    t2 = time.time()
    fb = fallback_from_smin(meta["s_min"])
    work = cal_dims[:, 0].astype(float) * cal_dims[:, 1] * cal_dims[:, 2]
    probs = predict_probs(theta, mean, std, Xc)
    thr = args.threshold
    table = None
    if thr <= 0:
        thr, table = choose_threshold(probs, cal_smin, work, fb)
    chosen = decide(probs, thr, fb)
    oracle_work = float(np.sum(work * np.minimum(cal_smin, fb) * (np.minimum(cal_smin, fb) + 1) / 2))
    fixed = {int(sf): float(np.sum(work * escalation_work(np.full(len(work), sf), cal_smin, fb)[0])) / oracle_work
             for sf in range(6, fb + 1)}
    write_model(args.out, theta, mean, std, thr, fb)
    rec = {"problems": args.problems, "sizes": [args.lo, args.hi], "phi_hi": args.phi_hi, "targets": list(TARGETS),
           "samples": int(train_mask.sum()), "data_s": t1 - t0, "train_s": t2 - t1, "final_loss": losses[-1],
           "first_loss": losses[0], "fallback": fb, "threshold": thr, "threshold_table": table,
           "calibration": {"problems": int(len(cal_smin)), "sizes": [args.cal_lo, args.cal_hi],
                           "phi_hi": args.cal_phi_hi, "target": args.cal_target, "seed": args.cal_seed,
                           "selector_eval": selector_eval(chosen, np.minimum(cal_smin, 17), work),
                           "work_vs_perfect_choice": float(np.sum(work * escalation_work(chosen, cal_smin, fb)[0]))
                           / oracle_work,
                           "fixed_count_work_vs_perfect_choice": fixed},
           "label_hist": np.bincount(y, minlength=N_CLASSES).tolist(),
           "s_min_hist": np.bincount(meta["s_min"], minlength=S_MEASURE + 2).tolist()}
    if args.record:
        with open(args.record, "w") as f:
            json.dump(rec, f)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
