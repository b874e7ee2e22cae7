#!/usr/bin/env python
"""Benchmark: FP64-equivalent GEMM TFLOP/s at <= 1e-12 componentwise error (relative to |A||B|)
of learned-slice batched emulation against fixed-slice emulation, on one GB300.

A step (the headline) is one ozg_dgemm_grouped call over a batch of 2048 uneven DGEMMs (m, n, k
log-uniform in [32, 2048], entries (u - 0.5) exp(phi g), phi ~ U(0, 4) per call) with slices = 0:
the learned selector (Sec. 4's adaptive split number) picks s per call for the 1e-12 target,
the split, the tensor-core slice products with the fused epilogue and the sampled double-double
check of every call run as one graph-replayed sequence of batched launches, and calls the
check rejects are re-run at the fallback count.  value = sum of 2 m n k over the batch / the
step time.

Beside it, in the same JSON line: the fixed-slice baselines on the same batch (s = 7 issued one
ozg_dgemm call at a time, and fixed counts in one grouped call, with the fraction of calls each
meets 1e-12 on), the native FP64 kernel, the 8192^3 DGEMM slice sweep (phi in {0.5, 2, 4},
s = 3..10, error and TFLOP/s per s), the KKR-like ZGEMM (n = 3616, s = 4..10), the roofline of
the grouped slice-product kernel, the CPU oracle on a bounded sample, and an end-to-end number
with the whole batch copied host -> device and the results device -> host in every step.

roofline.traffic is the per-launch DRAM bytes of the committed one-pass ncu summary under
profiles/ when it was taken on the current kernel sources (sha256 of ozg_gemm.cu,
ozg_device.cuh, ozg_internal.h and ozg_round.cuh), else null; a figure taken on other sources
is reported as roofline.traffic_other_source with the hash it was taken on.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ozg|reference]

Under torchrun every rank runs its own batch of the same distribution (independent problems,
no data-path collective: weak scaling); value = all ranks' flops / the slowest rank's time.
--impl reference times the CPU oracle doing the same method (features, selector, emulated
GEMM at the selected s) on a bounded sample of the batch (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64-equiv GEMM TFLOP/s at ≤1e-12 rel err: learned+batched vs fixed-slice"
TARGET_ERR = 1e-12
COUNT = 2048
BATCH_SEED = 4
CHECK_SAMPLES = 64
FIXED_SWEEP = (7, 9, 10, 11, 12)
SINGLE_PHIS = (0.5, 2.0, 4.0)
SELECTOR_MODEL = ""                 # set from --selector in main()
LABEL_SWEEP = tuple(range(5, 14))   # fixed counts whose sampled check labels each call's minimal s
ESCALATED_FIXED = (8, 9, 10)        # fixed counts run through the learned pipeline (same check, escalation)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ozg", choices=["ozg", "reference"])
    ap.add_argument("--count", type=int, default=COUNT, help="GEMMs in the batch")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the fixed-slice and native comparisons")
    ap.add_argument("--no-single", action="store_true", help="skip the 8192^3 slice sweep")
    ap.add_argument("--single-size", type=int, default=8192)
    ap.add_argument("--single-phis", default="0.5,2,4", help="phi values of the single-DGEMM sweep")
    ap.add_argument("--single-slices", default="3-10", help="slice counts of the single-DGEMM sweep (a-b or list)")
    ap.add_argument("--only-single", action="store_true", help="run only the single-DGEMM section (profiling)")
    ap.add_argument("--no-zgemm", action="store_true", help="skip the KKR-like ZGEMM section")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end number")
    ap.add_argument("--no-shim", action="store_true", help="skip the BLAS shim data-strategy section")
    ap.add_argument("--e2e-parts", type=int, default=E2E_PARTS, help="sub-batches of the device-buffer pipeline")
    ap.add_argument("--host-parts", type=int, default=HOST_PARTS, help="parts of the host-memory entry point")
    ap.add_argument("--shim-size", type=int, default=8192, help="n of the shim's n^3 DGEMM")
    ap.add_argument("--no-regions", action="store_true", help="skip the region-adaptive slice-count section")
    ap.add_argument("--selector", default="", help="selector model file (default: the package's model)")
    ap.add_argument("--tile-variant", type=int, default=-1,
                    help="force a tile variant of the slice-product kernel (default: autotuned)")
    args = ap.parse_args()
    if not args.selector:
        from paper_2503_22875_gb300 import selector
        args.selector = selector.DEFAULT_MODEL
    return args


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def world_max(pg, x: float, device) -> float:
    """Maximum of x over all ranks (the slowest rank's time), or x itself without a group."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def weak_value(flops_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job TFLOP/s: every rank's (equal-sized) batch over the slowest rank's step time."""
    return flops_per_rank * world / (ms_max / 1e3) / 1e12


def rank_batch_seed(rank: int) -> int:
    """Each rank draws its own batch (independent problems of the same distribution)."""
    return BATCH_SEED + rank


# ------------------------------------------------------------------------------------ peaks
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def source_hash():
    h = hashlib.sha256()
    for f in ("ozg_gemm.cu", "ozg_device.cuh", "ozg_internal.h", "ozg_round.cuh"):
        with open(os.path.join(ROOT, "paper_2503_22875_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profile_traffic(name: str):
    """(bytes, sha256 of the kernel sources it was taken on, tile variant or None) from the
    committed ncu summary profiles/<name>.md, or (None, None, None) when it is missing."""
    path = os.path.join(ROOT, "profiles", f"{name}.md")
    if not os.path.exists(path):
        return None, None, None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"source_sha256:\s*([0-9a-f]{64})", txt)
    v = re.search(r"tile_variant:\s*(\d+)", txt)
    return (float(m.group(1)) if m else None), (h.group(1) if h else None), (int(v.group(1)) if v else None)


def kernel_traffic(name: str, variant=None):
    """Per-launch DRAM bytes of the current kernel source, or None when the summary is missing,
    was taken on a different version of the kernel source or on another tile variant."""
    t, sha, v = profile_traffic(name)
    if variant is not None and v is not None and v != variant:
        return None
    return t if t is not None and sha == source_hash() else None


def stale_traffic(name: str, variant=None):
    """The last capture's figure when it was taken on other kernel sources or another tile
    variant (reported beside the null traffic, never as the traffic), else None."""
    t, sha, v = profile_traffic(name)
    if t is None or sha is None or (sha == source_hash() and (variant is None or v is None or v == variant)):
        return None
    return {"bytes_per_launch": t, "source_sha256": sha, "tile_variant": v, "profile": f"profiles/{name}.md"}


# slice-product kernel of a grouped launch, by tile variant
GROUPED_KERNELS = {0: "slice_gemm_grouped_kernel<256, 1>", 1: "slice_gemm_grouped_kernel<128, 2>",
                   2: "slice_gemm_grouped_kernel<256, 1>", 3: "slice_gemm_grouped_kernel<128, 1>",
                   4: "slice_gemm_pair_kernel", 5: "slice_gemm_grouped_stacked_kernel"}


def tensor_roofline(kernel, flops, ms, traffic_name, variant=None):
    """Roofline of a slice-product kernel: algorithmic tensor flops (s(s+1)/2 FP16 products of
    2 m n k each) over its CUDA-event duration, against the measured dense bf16 peak (FP16
    operands run at the same nominal rate).  The burst peak: each timed launch lasts well under
    a second and the sampled clocks stay at the maximum."""
    peaks, src = measured_peaks()
    peak = peaks.get("bf16_tflops")
    achieved = flops / (ms / 1e3) / 1e12
    return {"bound": "tensor", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": kernel_traffic(traffic_name, variant),
            "traffic_other_source": stale_traffic(traffic_name, variant),
            "peak_src": f"{src} bf16 burst (cuBLAS); sustained {peaks.get('bf16_tflops_sustained')}",
            "frac_of_sustained": achieved / peaks.get("bf16_tflops_sustained", peak),
            "tensor_flops_per_launch": flops, "launch_ms": ms}


# ------------------------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="ozg_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------------ CPU oracle
def oracle_sample(count, budget_s):
    """Calls of the batch taken in batch order while their estimated oracle time still fits
    budget_s (same shapes, spreads and per-call seeds; numpy draws), at most 64."""
    import oracle
    from paper_2503_22875_gb300 import selector, workloads
    oracle.build()
    model = selector.read_model(SELECTOR_MODEL)
    s_cap = max(model["s_lo"] + 10, model["fallback"])
    rate = 3.0e9  # int64 MACs per second of the threaded oracle (order of magnitude, for the budget)
    sample, est = [], 0.0
    for c in workloads.grouped_batch(count, seed=BATCH_SEED):
        cost = 60.0 * c.m * c.n * c.k / rate
        if est + cost > budget_s:
            continue
        A, B = workloads.call_matrices(c)
        sample.append((c, A, B))
        est += cost
        if len(sample) == 64:
            break
    return sample, model, s_cap


def oracle_step(sample, model, s_cap):
    """One pass of the method on the CPU oracle: features -> selector -> emulated GEMM."""
    import oracle
    t0 = time.perf_counter()
    flops = 0.0
    chosen = []
    for c, A, B in sample:
        f = oracle.features(A, B, TARGET_ERR)
        s, _ = oracle.mlp_select(model, f, s_cap)
        oracle.dgemm_emu(A, B, s)
        flops += 2.0 * c.m * c.n * c.k
        chosen.append(s)
    return time.perf_counter() - t0, flops, chosen


def cpu_baseline(count, budget_s=12.0):
    import oracle
    sample, model, s_cap = oracle_sample(count, budget_s)
    dt, flops, chosen = oracle_step(sample, model, s_cap)
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": (f"{len(sample)} GEMMs of the {count}-GEMM batch (taken in batch order while the estimated "
                       f"time fits {budget_s:g} s; numpy draws of the same shapes and spreads, "
                       f"{sum(2.0 * c.m * c.n * c.k for c, _, _ in sample) / 1e9:.1f} GFLOP): oracle features, "
                       f"oracle selector (FP32 emulation of the same model), oracle emulated DGEMM at the selected s "
                       f"(chosen {sorted(set(chosen))}); {dt:.1f} s")}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    import oracle
    sample, model, s_cap = oracle_sample(args.count, 6.0)
    for _ in range(args.warmup):
        oracle_step(sample, model, s_cap)
    tot_t, tot_f = 0.0, 0.0
    for _ in range(args.steps):
        dt, fl, chosen = oracle_step(sample, model, s_cap)
        tot_t += dt
        tot_f += fl
    val = tot_f / tot_t / 1e12
    ms = 1e3 * tot_t / args.steps
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"learned-slice emulated DGEMM on {len(sample)} GEMMs of the "
                                   f"{args.count}-GEMM batch (m,n,k log-uniform [32,2048], phi~U(0,4)), target "
                                   f"{TARGET_ERR:g}; CPU oracle", "calls": len(sample), "target": TARGET_ERR},
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": oracle.threads(), "kind": "oracle",
                             "sample": (f"{len(sample)} GEMMs of the batch per step (batch order, within a 6 s "
                                        f"estimate), features + selector + emulated DGEMM")},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------ helpers
def timed(torch, st, fn, steps, warm=1):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(steps):
            fn()
        e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def report_stats(reps):
    errs = np.array([r.est_err for r in reps], dtype=float)
    used = [r.slices_used for r in reps]
    return {"frac_le_target": float(np.mean(errs <= TARGET_ERR)), "max_err_sampled_dd": float(np.nanmax(errs)),
            "slices_hist": {int(v): int(c) for v, c in zip(*np.unique(used, return_counts=True))}}


def tensor_flops(batch, slices):
    return sum(s * (s + 1) / 2 * 2.0 * c.m * c.n * c.k for c, s in zip(batch.calls, slices))


# ------------------------------------------------------------------------------------ comparisons
def pass_products(reps, fallback):
    """Slice products of every pass each learned call ran: the selected count, then each re-run."""
    from paper_2503_22875_gb300 import selector
    return [sum(x * (x + 1) / 2 for x in selector.escalation_passes(r.selected, r.repaired, fallback)) for r in reps]


def escalated_policy(ozg, torch, calls, flops, st, steps, model_path, work):
    """A learned-pipeline policy on the batch: CUDA-event time per step and what the check did."""
    from paper_2503_22875_gb300 import selector
    n = len(calls)
    ctx = ozg.Context(stream=st)
    ctx.load_selector(model_path)
    ctx.set_target_error(TARGET_ERR)
    ctx.set_check_samples(CHECK_SAMPLES)
    ms = timed(torch, st, lambda: ctx.dgemm_grouped(calls, [0] * n), max(1, min(steps, 5)))
    with torch.cuda.stream(st):
        reps = ctx.dgemm_grouped(calls, [0] * n, report=True)
    ctx.close()
    fb = selector.read_model(model_path)["fallback"]
    prods = pass_products(reps, fb)
    out = {"ms": ms, "tflops": flops / (ms / 1e3) / 1e12, **report_stats(reps),
           "reruns_1": int(sum(r.repaired == 1 for r in reps)), "reruns_2": int(sum(r.repaired >= 2 for r in reps)),
           "tensor_products_work": float(np.dot(prods, work))}
    return out, reps


def compare_section(ozg, torch, batch, calls, flops, st, steps, learned_reps):
    """Fixed-slice baselines and the native FP64 kernel on the same batch; per-call minimal counts
    from the sampled check at fixed counts; fixed counts through the learned pipeline."""
    from paper_2503_22875_gb300 import selector
    out = {}
    n = len(calls)
    work = np.array([float(c.m) * c.n * c.k for c in batch.calls])
    # per-call labels: the smallest fixed count whose 64-sample check meets the target
    ctx = ozg.Context(stream=st)
    ctx.set_check_samples(CHECK_SAMPLES)
    smin = np.full(n, LABEL_SWEEP[-1] + 1)
    for s in reversed(LABEL_SWEEP):
        with torch.cuda.stream(st):
            reps = ctx.dgemm_grouped(calls, [s] * n, report=True)
        ok = np.array([r.est_err <= TARGET_ERR for r in reps])
        smin[ok] = s
    ctx.close()
    out["minimal_s_hist"] = {int(v): int(c) for v, c in zip(*np.unique(smin, return_counts=True))}
    fb = selector.read_model(SELECTOR_MODEL)["fallback"]
    perfect = float(np.dot(work, np.minimum(smin, fb) * (np.minimum(smin, fb) + 1) / 2))
    learned_work = float(np.dot(pass_products(learned_reps, fb), work))
    sel_eval = selector.selector_eval([r.selected for r in learned_reps], smin, work)
    sel_eval["labels"] = (f"per call, the smallest s in {LABEL_SWEEP[0]}..{LABEL_SWEEP[-1]} whose {CHECK_SAMPLES}-sample "
                          f"GPU check (exact reference) meets {TARGET_ERR:g} in a fixed-count grouped run")
    sel_eval["tensor_work_vs_perfect_choice"] = learned_work / perfect
    esc = {}
    with tempfile.TemporaryDirectory() as tmp:
        for s in ESCALATED_FIXED + (fb,):
            path = os.path.join(tmp, f"const{s}.ozgsel")
            selector.write_constant_model(path, s, fb)
            res, _ = escalated_policy(ozg, torch, calls, flops, st, steps, path, work)
            res["tensor_work_vs_perfect_choice"] = res.pop("tensor_products_work") / perfect
            esc[s] = res
    out["fixed_escalated"] = esc
    out["fixed_escalated_note"] = (f"fixed s through the learned pipeline (the same feature pass, {CHECK_SAMPLES}-sample "
                                   f"check and escalation: a rejected call re-runs at min(s + 2, {fb}), then at {fb})")
    ctx = ozg.Context(stream=st)
    ms = timed(torch, st, lambda: [ctx.dgemm(*c, 7) for c in calls], max(1, min(steps, 2)))
    ctx.set_check_samples(CHECK_SAMPLES)
    with torch.cuda.stream(st):
        reps = [ctx.dgemm(*c, 7, report=True) for c in calls]
    out["fixed_s7_one_at_a_time"] = {"ms": ms, "tflops": flops / (ms / 1e3) / 1e12, "check": "none while timed",
                                     **report_stats(reps)}
    ctx.close()
    fixed = {}
    for s in FIXED_SWEEP:
        # timed with the same per-call sampled check the learned step runs (and without it)
        ctx = ozg.Context(stream=st)
        ms_nocheck = timed(torch, st, lambda: ctx.dgemm_grouped(calls, [s] * n), max(1, min(steps, 5)))
        ctx.close()
        ctx = ozg.Context(stream=st)
        ctx.set_check_samples(CHECK_SAMPLES)
        ms = timed(torch, st, lambda: ctx.dgemm_grouped(calls, [s] * n), max(1, min(steps, 5)))
        with torch.cuda.stream(st):
            reps = ctx.dgemm_grouped(calls, [s] * n, report=True)
        fixed[s] = {"ms": ms, "tflops": flops / (ms / 1e3) / 1e12, "tflops_without_check": flops / (ms_nocheck / 1e3) / 1e12,
                    **report_stats(reps)}
        ctx.close()
    out["fixed_grouped"] = fixed
    ok_all = [s for s in FIXED_SWEEP if fixed[s]["frac_le_target"] >= 1.0]
    ok_99 = [s for s in FIXED_SWEEP if fixed[s]["frac_le_target"] >= 0.99]
    out["smallest_fixed_s_meeting_target_on_all_calls"] = min(ok_all) if ok_all else None
    out["smallest_fixed_s_meeting_target_on_99pct"] = min(ok_99) if ok_99 else None
    # the learned step with each tile variant forced, against the autotuned choice
    tv = {}
    for v in range(6):
        ctx = ozg.Context(stream=st)
        ctx.load_selector(SELECTOR_MODEL)
        ctx.set_target_error(TARGET_ERR)
        ctx.set_check_samples(CHECK_SAMPLES)
        ctx.set_tile_variant(v)
        tv[v] = timed(torch, st, lambda: ctx.dgemm_grouped(calls, [0] * n), max(1, min(steps, 5)))
        ctx.close()
    out["learned_ms_by_tile_variant"] = tv
    ctx = ozg.Context(stream=st)
    ms = timed(torch, st, lambda: [ctx.native_dgemm(*c) for c in calls], 1, warm=0)
    out["native_fp64_one_at_a_time"] = {"ms": ms, "tflops": flops / (ms / 1e3) / 1e12}
    ctx.close()
    return out, sel_eval


def parse_list(spec, cast):
    if "-" in spec and "," not in spec:
        a, b = spec.split("-")
        return list(range(int(a), int(b) + 1))
    return [cast(x) for x in spec.split(",")]


def shim_section(torch, n, reps=3):
    """The BLAS interposition library's three data strategies (Sec. 2.1) on an n^3 DGEMM called
    through dgemm_ on arrays in pageable host memory, at s = 7: wall-clock time of each
    synchronous call.  copy: DMA from and to the caller's arrays; coherent: the kernels read and write
    the host arrays in place over the CPU-GPU link; migrate: the first call moves the arrays'
    pages to GPU memory, later calls find them there."""
    import ctypes

    from paper_2503_22875_gb300 import build
    lib = ctypes.CDLL(build.SHIM_LIB)
    lib.ozg_blas_set_mode.argtypes = [ctypes.c_int]
    lib.ozg_blas_set_strategy.argtypes = [ctypes.c_int]
    lib.ozg_blas_migrated_bytes.restype = ctypes.c_longlong
    gen = torch.Generator(device="cuda")
    gen.manual_seed(77)

    def draw():  # a = (u - 0.5) exp(0.5 g), drawn on the GPU, returned in pageable host memory
        u = torch.rand((n, n), generator=gen, device="cuda", dtype=torch.float64)
        z = torch.randn((n, n), generator=gen, device="cuda", dtype=torch.float64)
        return ((u - 0.5) * torch.exp(0.5 * z)).cpu().numpy()
    A, B = draw(), draw()
    torch.cuda.empty_cache()
    ci, cd = ctypes.c_int, ctypes.c_double
    one, zero, nn = cd(1.0), cd(0.0), ci(n)

    def call(C):
        lib.dgemm_(b"N", b"N", ctypes.byref(nn), ctypes.byref(nn), ctypes.byref(nn), ctypes.byref(one),
                   ctypes.c_void_p(A.ctypes.data), ctypes.byref(nn), ctypes.c_void_p(B.ctypes.data), ctypes.byref(nn),
                   ctypes.byref(zero), ctypes.c_void_p(C.ctypes.data), ctypes.byref(nn), ctypes.c_size_t(1),
                   ctypes.c_size_t(1))
    names = {0: "copy", 1: "coherent", 2: "migrate"}
    out = {"workload": f"dgemm_ {n}^3 through libozg_blas.so on pageable host arrays, OZG_COMPUTE_MODE=fp64_int8_7, "
                       "beta = 0, wall-clock per synchronous call", "slices": 7}
    lib.ozg_blas_set_mode(7)
    flops = 2.0 * n ** 3
    for st, name in names.items():
        lib.ozg_blas_set_strategy(st)
        C = np.zeros((n, n))
        times = []
        for _ in range(reps + 1):
            t0 = time.perf_counter()
            call(C)
            times.append(time.perf_counter() - t0)
        steady = float(np.median(times[1:]))
        entry = {"strategy_in_effect": names.get(lib.ozg_blas_get_strategy(), "?"), "first_call_ms": times[0] * 1e3,
                 "steady_ms": steady * 1e3, "steady_tflops": flops / steady / 1e12}
        if st == 2:
            entry["migrated_bytes"] = int(lib.ozg_blas_migrated_bytes())
        out[name] = entry
    lib.ozg_blas_set_strategy(0)
    return out


def regions_section(ozg, torch, n, steps, cases=((0.5, 4.0), (0.1, 6.0)), bands=(4, 8)):
    """Region-adaptive slice counts (the paper's Sec. 4 proposal): n^3 DGEMMs whose first quarter
    of the rows of A has exponent spread phi_wide and the rest phi (B: phi), per (phi, phi_wide)
    case.  One learned call on the whole matrix (one count for all of C) against row bands whose
    counts the selector picks per region (ozg_dgemm_regions); target 1e-12, the 64-sample check
    judging every call or region (a rejected one is re-run at the fallback count), graph-replayed,
    CUDA events."""
    st = torch.cuda.Stream()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(91)

    def draw(rows, cols, p):
        u = torch.rand((rows, cols), generator=gen, device="cuda", dtype=torch.float64)
        z = torch.randn((rows, cols), generator=gen, device="cuda", dtype=torch.float64)
        return (u - 0.5) * torch.exp(p * z)
    flops = 2.0 * n ** 3
    out = {"workload": f"DGEMM {n}^3, rows 0..{n // 4 - 1} of A with a=(u-0.5)exp(phi_wide g), the other rows and "
                       f"B with exp(phi g); target {TARGET_ERR:g}, {CHECK_SAMPLES}-sample check per call or region",
           "cases": []}
    dC = torch.empty((n, n), dtype=torch.float64, device="cuda")
    for phi, phi_wide in cases:
        # column-major n x n: row i of A is column i of the row-major tensor
        dA = draw(n, n, phi)
        dA[:, : n // 4] = draw(n, n // 4, phi_wide)
        dB = draw(n, n, phi)
        ctx = ozg.Context(stream=st)
        ctx.load_selector(SELECTOR_MODEL)
        ctx.set_target_error(TARGET_ERR)
        ctx.set_check_samples(CHECK_SAMPLES)
        case = {"phi": phi, "phi_wide": phi_wide}
        with torch.cuda.stream(st):
            rep = ctx.dgemm("N", "N", n, n, n, 1.0, dA, n, dB, n, 0.0, dC, n, 0, report=True)
        ms = timed(torch, st, lambda: ctx.dgemm("N", "N", n, n, n, 1.0, dA, n, dB, n, 0.0, dC, n, 0), steps)
        case["whole_matrix"] = {"ms": ms, "tflops": flops / (ms / 1e3) / 1e12, "selected": rep.selected,
                                "slices_used": rep.slices_used, "repaired": rep.repaired,
                                "err_sampled_dd": rep.est_err}
        for b in bands:
            with torch.cuda.stream(st):
                reps = ctx.dgemm_regions("N", "N", n, n, n, 1.0, dA, n, dB, n, 0.0, dC, n, b, 1, report=True)
            ms = timed(torch, st,
                       lambda: ctx.dgemm_regions("N", "N", n, n, n, 1.0, dA, n, dB, n, 0.0, dC, n, b, 1), steps)
            case[f"row_bands_{b}"] = {"ms": ms, "tflops": flops / (ms / 1e3) / 1e12,
                                      "selected": [r.selected for r in reps],
                                      "slices_used": [r.slices_used for r in reps],
                                      "max_err_sampled_dd": max(r.est_err for r in reps)}
        ctx.close()
        out["cases"].append(case)
        del dA, dB
    return out


def single_section(ozg, torch, size, steps, phis=SINGLE_PHIS, slice_list=tuple(range(3, 11))):
    """Config 2: emulated DGEMM size^3, a = (u - 0.5) exp(phi g), phi in {0.5, 2, 4}, s = 3..10:
    TFLOP/s and sampled double-double error per s, the native FP64 kernel, and the roofline of the
    slice-product kernel at phi = 0.5 with the smallest s meeting 1e-12."""
    n = size
    st = torch.cuda.Stream()
    gen = torch.Generator(device="cuda")
    dC = torch.empty((n, n), dtype=torch.float64, device="cuda")
    flops = 2.0 * n ** 3
    out = {"workload": f"emulated DGEMM {n}^3, a=(u-0.5)exp(phi g), u~U(0,1), g~N(0,1); GPU-drawn (seeded)",
           "by_phi": {}}
    roof = None
    for phi in phis:
        gen.manual_seed(int(1000 * phi) + 2)

        def draw():
            u = torch.rand((n, n), generator=gen, device="cuda", dtype=torch.float64)
            z = torch.randn((n, n), generator=gen, device="cuda", dtype=torch.float64)
            return (u - 0.5) * torch.exp(phi * z)
        dA, dB = draw(), draw()
        ctx = ozg.Context(stream=st)
        res = {}
        for s in slice_list:
            ctx.set_check_samples(0)
            ms = timed(torch, st, lambda: ctx.dgemm("N", "N", n, n, n, 1.0, dA, n, dB, n, 0.0, dC, n, s),
                       max(1, min(steps, 3)))
            ctx.set_check_samples(CHECK_SAMPLES)
            with torch.cuda.stream(st):
                rep = ctx.dgemm("N", "N", n, n, n, 1.0, dA, n, dB, n, 0.0, dC, n, s, report=True)
            res[s] = {"ms": ms, "tflops": flops / (ms / 1e3) / 1e12, "err_sampled_dd": rep.est_err}
        ok = [s for s in res if res[s]["err_sampled_dd"] <= TARGET_ERR]
        entry = {"by_slices": res, "smallest_s_meeting_target": min(ok) if ok else None}
        if phi == phis[0]:
            s = entry["smallest_s_meeting_target"] or 7
            ctx.set_check_samples(0)
            ctx.set_profiling(True)
            with torch.cuda.stream(st):
                for _ in range(max(3, min(steps, 5))):
                    ctx.dgemm("N", "N", n, n, n, 1.0, dA, n, dB, n, 0.0, dC, n, s)
            ph = ctx.phase_times()
            ctx.set_profiling(False)
            gemm_ms = ph["gemm"][0] / max(ph["gemm"][1], 1)
            # single calls of at most 16 slices run the stacked group-pair kernel (variant 5)
            kname = "slice_gemm_stacked_kernel" if s <= 16 else "slice_gemm_kernel"
            roof = tensor_roofline(kname, s * (s + 1) / 2 * flops, gemm_ms, f"slice_gemm_{n}_s{s}", 5 if s <= 16 else None)
            roof["slices"] = s
            roof["algorithmic_bytes"] = 2.0 * s * 2 * n * n + 8.0 * n * n
            ms_nat = timed(torch, st, lambda: ctx.native_dgemm("N", "N", n, n, n, 1.0, dA, n, dB, n, 0.0, dC, n), 1,
                           warm=0)
            entry["native_fp64_tflops"] = flops / (ms_nat / 1e3) / 1e12
        out["by_phi"][phi] = entry
        ctx.close()
        del dA, dB
    out["roofline_phi0.5"] = roof
    return out


def zgemm_section(ozg, torch, steps):
    """KKR-like complex128 ZGEMM, n = 113 x 32 = 3616 (stand-in for the MuST ZGEMMs of Sec. 3.2):
    emulated at s = 4..10 (FP64-equivalent 8 n^3 flops) with the sampled double-double error
    (|A||B|-relative, and the paper's per-part max_real / max_imag), and the native FP64 kernel."""
    from paper_2503_22875_gb300 import workloads
    A, B = workloads.kkr_like_pair(113, 32, seed=3)
    n = A.shape[0]
    dA, dB = ozg.to_device(A), ozg.to_device(B)
    dC = torch.empty((n, n), dtype=torch.complex128, device="cuda")
    st = torch.cuda.Stream()
    ctx = ozg.Context(stream=st)
    flops = 8.0 * n ** 3
    out = {"workload": f"KKR-like ZGEMM n={n} (113 blocks of 32), complex normal x exp(-|r_i - r_j|) + (1+0.1i) diag",
           "by_slices": {}}
    for s in range(4, 11):
        ctx.set_check_samples(0)
        ms = timed(torch, st, lambda: ctx.zgemm("N", "N", n, n, n, 1.0, dA, n, dB, n, 0.0, dC, n, s), steps)
        ctx.set_check_samples(CHECK_SAMPLES)
        with torch.cuda.stream(st):
            rep = ctx.zgemm("N", "N", n, n, n, 1.0, dA, n, dB, n, 0.0, dC, n, s, report=True)
        out["by_slices"][s] = {"ms": ms, "tflops": flops / (ms / 1e3) / 1e12, "err_sampled_dd": rep.est_err,
                               "max_real": rep.max_real, "max_imag": rep.max_imag}
    ok = [s for s, v in out["by_slices"].items() if v["err_sampled_dd"] <= TARGET_ERR]
    out["smallest_s_meeting_target"] = min(ok) if ok else None
    ms = timed(torch, st, lambda: ctx.native_zgemm("N", "N", n, n, n, 1.0, dA, n, dB, n, 0.0, dC, n), 1, warm=0)
    out["native_fp64_tflops"] = flops / (ms / 1e3) / 1e12
    # the variant whose diagonal shift puts cond_2(A) near 1e8 (shift found once on the host, cached)
    Ak, _ = workloads.kkr_kappa_pair(113, 32, seed=3, kappa=1e8)
    dAk = ozg.to_device(Ak)
    ctx.set_check_samples(CHECK_SAMPLES)
    kap = {}
    for s in range(4, 11):
        with torch.cuda.stream(st):
            rep = ctx.zgemm("N", "N", n, n, n, 1.0, dAk, n, dB, n, 0.0, dC, n, s, report=True)
        kap[s] = {"err_sampled_dd": rep.est_err, "max_real": rep.max_real, "max_imag": rep.max_imag}
    okk = [s for s, v in kap.items() if v["err_sampled_dd"] <= TARGET_ERR]
    out["kappa1e8"] = {"shift": str(workloads.kkr_kappa_shift(113, 32, 3, 1e8)), "by_slices": kap,
                       "smallest_s_meeting_target": min(okk) if okk else None}
    # 3M: three real emulated products (3/4 of the slice-product work, the 3M error bound)
    z3 = {}
    for s in range(5, 11):
        ctx.set_check_samples(0)
        ms = timed(torch, st, lambda: ctx.zgemm3m("N", "N", n, n, n, 1.0, dA, n, dB, n, 0.0, dC, n, s), steps)
        ctx.set_check_samples(CHECK_SAMPLES)
        with torch.cuda.stream(st):
            rep = ctx.zgemm3m("N", "N", n, n, n, 1.0, dA, n, dB, n, 0.0, dC, n, s, report=True)
        z3[s] = {"ms": ms, "tflops": flops / (ms / 1e3) / 1e12, "err_sampled_dd": rep.est_err,
                 "max_real": rep.max_real, "max_imag": rep.max_imag}
    ok3 = [s for s, v in z3.items() if v["err_sampled_dd"] <= TARGET_ERR]
    out["3m"] = {"by_slices": z3, "smallest_s_meeting_target": min(ok3) if ok3 else None}
    ctx.close()
    return out


E2E_PARTS = 4        # parts of the device-buffer pipeline (cross-step overlap)
HOST_PARTS = 16      # parts of ozg_dgemm_grouped_host (a synchronous call: fill and drain per step)


def e2e_pipelined(ozg, torch, batch, make_ctx, steps, pg, world, flops, nparts=E2E_PARTS):
    """End to end with host buffers: pinned host copies of A, B and C; per step, for every part,
    H2D of its A and B on one copy stream, the learned grouped call on the part's own stream,
    D2H of its C on another copy stream, ordered by events (a part's buffers are reused only after
    the previous step is done with them)."""
    n = len(batch.calls)
    w = np.cumsum([2.0 * c.m * c.n * c.k for c in batch.calls])
    cuts = [0] + [int(np.searchsorted(w, w[-1] * (i + 1) / nparts)) + 1 for i in range(nparts - 1)] + [n]
    cuts = sorted(set(min(max(x, 0), n) for x in cuts))
    calls = batch.gemm_calls()

    def rng(off, i, total):
        return off[cuts[i]], (off[cuts[i + 1]] if cuts[i + 1] < n else total)

    parts = []
    hA = torch.empty(batch.A.numel(), dtype=torch.float64, pin_memory=True)
    hB = torch.empty(batch.B.numel(), dtype=torch.float64, pin_memory=True)
    hC = torch.empty(batch.C.numel(), dtype=torch.float64, pin_memory=True)
    hA.copy_(batch.A)
    hB.copy_(batch.B)
    for i in range(len(cuts) - 1):
        a0, a1 = rng(batch.offA, i, batch.A.numel())
        b0, b1 = rng(batch.offB, i, batch.B.numel())
        c0, c1 = rng(batch.offC, i, batch.C.numel())
        st = torch.cuda.Stream()
        ctx = make_ctx()
        ctx.set_stream(st)
        parts.append({"calls": calls[cuts[i]:cuts[i + 1]], "st": st, "ctx": ctx, "A": (a0, a1), "B": (b0, b1),
                      "C": (c0, c1), "ev_in": torch.cuda.Event(), "ev_done": torch.cuda.Event(),
                      "ev_out": torch.cuda.Event()})
    h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(2, steps // 2)
    for it in range(1 + e2e_steps):
        if it == 1:
            torch.cuda.synchronize()
            e0.record(h2d)
        for P in parts:
            (a0, a1), (b0, b1), (c0, c1) = P["A"], P["B"], P["C"]
            if it > 0:
                h2d.wait_event(P["ev_done"])
            with torch.cuda.stream(h2d):
                batch.A[a0:a1].copy_(hA[a0:a1], non_blocking=True)
                batch.B[b0:b1].copy_(hB[b0:b1], non_blocking=True)
                P["ev_in"].record(h2d)
            P["st"].wait_event(P["ev_in"])
            if it > 0:
                P["st"].wait_event(P["ev_out"])
            P["ctx"].dgemm_grouped(P["calls"], [0] * len(P["calls"]))
            P["ev_done"].record(P["st"])
            d2h.wait_event(P["ev_done"])
            with torch.cuda.stream(d2h):
                hC[c0:c1].copy_(batch.C[c0:c1], non_blocking=True)
                P["ev_out"].record(d2h)
    e1.record(d2h)
    e1.synchronize()
    ms = world_max(pg, e0.elapsed_time(e1) / e2e_steps, "cuda")
    for P in parts:
        P["ctx"].close()
    del hA, hB, hC
    return {"value": weak_value(flops, world, ms), "unit": "TFLOP/s",
            "h2d_bytes_per_step": 8 * (batch.A.numel() + batch.B.numel()),
            "d2h_bytes_per_step": 8 * batch.C.numel(), "ms_per_step": ms,
            "pipeline": f"{len(parts)} sub-batches, H2D / compute / D2H overlapped on separate streams"}


def e2e_host_abi(ozg, torch, batch, make_ctx, steps, pg, world, flops, nparts=HOST_PARTS):
    """End to end through the host-memory C ABI: the batch lives in pinned host memory (each
    call's A, B and C back to back in three buffers) and every step is one synchronous
    ozg_dgemm_grouped_host call -- the library copies the inputs in, computes the learned grouped
    emulation in pipelined parts and copies C out.  Wall-clock per call (the call returns when C
    is on the host), after one untimed call that builds the parts' plans."""
    calls = batch.calls
    n = len(calls)
    sz = {"A": [c.m * c.k for c in calls], "B": [c.k * c.n for c in calls], "C": [c.m * c.n for c in calls]}
    host, offs = {}, {}
    for key, dev in (("A", batch.A), ("B", batch.B), ("C", batch.C)):
        o = np.concatenate([[0], np.cumsum(sz[key])]).astype(np.int64)
        offs[key] = o
        host[key] = torch.empty(int(o[-1]), dtype=torch.float64, pin_memory=True)
        if key != "C":
            src = {"A": batch.offA, "B": batch.offB}[key]
            packed = torch.cat([dev[src[i]:src[i] + sz[key][i]] for i in range(n)])
            host[key].copy_(packed)
            del packed
    torch.cuda.empty_cache()
    ptr = {key: host[key].data_ptr() for key in host}
    descs = [("N", "N", c.m, c.n, c.k, 1.0, ptr["A"] + 8 * int(offs["A"][i]), c.m, ptr["B"] + 8 * int(offs["B"][i]),
              c.k, 0.0, ptr["C"] + 8 * int(offs["C"][i]), c.m) for i, c in enumerate(calls)]
    ctx = make_ctx()
    ctx.set_host_parts(nparts)
    ctx.dgemm_grouped_host(descs, [0] * n)  # plans and graphs of the parts
    e2e_steps = max(2, steps // 2)
    if pg is not None:
        pg.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.dgemm_grouped_host(descs, [0] * n)
    ms = world_max(pg, (time.perf_counter() - t0) * 1e3 / e2e_steps, "cuda")
    reps = ctx.dgemm_grouped_host(descs, [0] * n, report=True)
    ctx.close()
    out = {"value": weak_value(flops, world, ms), "unit": "TFLOP/s",
           "h2d_bytes_per_step": 8 * (int(offs["A"][-1]) + int(offs["B"][-1])),
           "d2h_bytes_per_step": 8 * int(offs["C"][-1]), "ms_per_step": ms,
           "api": f"ozg_dgemm_grouped_host (host pointers in, C on the host out; {nparts} pipelined parts)",
           "frac_le_target": float(np.mean([r.est_err <= TARGET_ERR for r in reps]))}
    del host
    return out


# ------------------------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch

    from paper_2503_22875_gb300 import build, ozg, workloads

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if args.only_single:
        build.build()
        ozg.load()
        sec = single_section(ozg, torch, args.single_size, args.steps, parse_list(args.single_phis, float),
                             parse_list(args.single_slices, int))
        print(json.dumps({"single_dgemm": sec}), flush=True)
        return 0
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    # rank 0 compiles if anything is stale; the others wait and then find the library up to date
    # (concurrent builds would write the same object files)
    if pg is None or rank == 0:
        build.build()
    if pg is not None:
        pg.barrier()
        if rank != 0:
            build.build()
    ozg.load()
    batch = workloads.grouped_batch_flat(args.count, seed=rank_batch_seed(rank))
    calls = batch.gemm_calls()
    n = len(calls)
    flops = sum(2.0 * c.m * c.n * c.k for c in batch.calls)
    in_bytes = 8 * (batch.A.numel() + batch.B.numel())
    st = torch.cuda.Stream()
    torch.cuda.synchronize()

    def learned_ctx():
        c = ozg.Context(stream=st)
        c.load_selector(SELECTOR_MODEL)
        c.set_target_error(TARGET_ERR)
        c.set_check_samples(CHECK_SAMPLES)
        if args.tile_variant >= 0:
            c.set_tile_variant(args.tile_variant)
        else:
            c.set_autotune(True)  # the batch's tile variant, timed once per batch and cached
        return c

    ctx = learned_ctx()
    auto = [0] * n
    with torch.cuda.stream(st):
        ctx.dgemm_grouped(calls, auto)  # plan (tile variant autotuned), digit workspace, graph capture
        for _ in range(args.warmup):
            ctx.dgemm_grouped(calls, auto)
    torch.cuda.synchronize()
    tile_variant = ctx.tile_variant()
    clocks = ClockSampler(local)
    if pg is not None:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    l0 = ozg.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        e0.record(st)
        for _ in range(args.steps):
            ctx.dgemm_grouped(calls, auto)
        e1.record(st)
    e1.synchronize()
    launches = ozg.kernel_launches() - l0
    clk = clocks.stop()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = world_max(pg, ms, "cuda")
    value = weak_value(flops, world, ms_max)
    with torch.cuda.stream(st):
        reps = ctx.dgemm_grouped(calls, auto, report=True)
    stats = report_stats(reps)
    used = [r.slices_used for r in reps]
    stats["selected_hist"] = {int(v): int(c) for v, c in zip(*np.unique([r.selected for r in reps],
                                                                           return_counts=True))}
    stats["repaired"] = int(sum(r.repaired > 0 for r in reps))
    stats["reruns"] = {"at_s_plus_2": int(sum(r.repaired == 1 for r in reps)),
                       "then_at_fallback": int(sum(r.repaired >= 2 for r in reps))}
    # tensor work of the step: every call at its selected count, plus the escalated re-runs
    from paper_2503_22875_gb300 import selector
    fallback = selector.read_model(SELECTOR_MODEL)["fallback"]
    tflops_step = sum(p * 2.0 * c.m * c.n * c.k for p, c in zip(pass_products(reps, fallback), batch.calls))

    # the slice-product kernel's own duration: the same step without the graph, CUDA events
    # around each grouped GEMM launch on the launch stream
    pctx = learned_ctx()
    pctx.set_graphs(False)
    with torch.cuda.stream(st):
        pctx.dgemm_grouped(calls, auto)
    pctx.set_profiling(True)
    pctx.phase_times()
    rsteps = max(3, min(args.steps, 5))
    with torch.cuda.stream(st):
        for _ in range(rsteps):
            pctx.dgemm_grouped(calls, auto)
    ph = pctx.phase_times()
    pctx.close()
    gemm_ms = ph["gemm"][0] / rsteps
    grouped_ms_nograph = ph["grouped"][0] / max(ph["grouped"][1], 1)
    roof = tensor_roofline(GROUPED_KERNELS.get(tile_variant, "slice_gemm_grouped_kernel"), tflops_step, gemm_ms,
                           f"slice_gemm_grouped_learned_{n}", tile_variant)
    # algorithmic DRAM bytes of the launch: each selected digit plane read once, C written once
    roof["algorithmic_bytes"] = sum(2.0 * r.selected * (c.m + c.n) * c.k + 8.0 * c.m * c.n
                                    for c, r in zip(batch.calls, reps))
    roof["note"] = ("tensor flops = sum over calls of s(s+1)/2 * 2mnk at the selected s (plus escalated re-runs); "
                    "launch_ms = the step's grouped GEMM launches, CUDA events, without the graph")

    # end to end through the host-memory C ABI (ozg_dgemm_grouped_host): every step copies the
    # whole batch host -> device, runs it and copies C back, pipelined in HOST_PARTS parts inside
    # the library; beside it, the same with torch copies into device buffers and the device entry
    e2e = None
    if not args.no_e2e:
        e2e = e2e_host_abi(ozg, torch, batch, learned_ctx, args.steps, pg, world, flops, args.host_parts)
        e2e["device_buffer_pipeline"] = e2e_pipelined(ozg, torch, batch, learned_ctx, args.steps, pg, world, flops,
                                                      args.e2e_parts)
    ctx.close()
    if pg is not None:
        pg.barrier()

    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return 0

    compare = None
    sel_eval = None
    if not args.no_compare:
        compare, sel_eval = compare_section(ozg, torch, batch, calls, flops, st, args.steps, reps)
        learned = value / world
        compare["learned_vs_fixed_s7_one_at_a_time"] = learned / compare["fixed_s7_one_at_a_time"]["tflops"]
        best = compare["smallest_fixed_s_meeting_target_on_all_calls"]
        if best:
            compare["learned_vs_smallest_sufficient_fixed_grouped"] = learned / compare["fixed_grouped"][best]["tflops"]
        esc = compare["fixed_escalated"]
        ok = {s: v for s, v in esc.items() if v["frac_le_target"] >= 1.0}
        if ok:
            s_best = max(ok, key=lambda s: ok[s]["tflops"])
            compare["best_fixed_escalated"] = s_best
            compare["learned_vs_best_fixed_escalated"] = learned / ok[s_best]["tflops"]
        fbk = max(esc)
        compare["learned_vs_fixed_fallback"] = learned / esc[fbk]["tflops"]
        compare["learned_vs_native_fp64"] = learned / compare["native_fp64_one_at_a_time"]["tflops"]
    del batch, calls
    torch.cuda.empty_cache()
    single = None if args.no_single else single_section(ozg, torch, args.single_size, args.steps,
                                                        parse_list(args.single_phis, float),
                                                        parse_list(args.single_slices, int))
    zgemm = None if args.no_zgemm else zgemm_section(ozg, torch, max(1, min(args.steps, 3)))
    regions = None if args.no_regions else regions_section(ozg, torch, args.single_size, max(1, min(args.steps, 3)))
    shim = None if (world > 1 or args.no_shim) else shim_section(torch, args.shim_size)
    cpu = None if (world > 1 or args.no_cpu_baseline) else cpu_baseline(args.count)

    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 (int8-range digits in fp16 on tcgen05, exact integer accumulation)",
        "data": "synthetic",
        "config": {"workload": (f"learned+batched: {n} DGEMMs (m,n,k log-uniform [32,2048], a=(u-0.5)exp(phi g), "
                                f"phi~U(0,4) per call, beta=0), slices chosen per call by the selector MLP for "
                                f"{TARGET_ERR:g}, one graph-replayed ozg_dgemm_grouped call per step"),
                   "calls": n, "target": TARGET_ERR, "check_samples": CHECK_SAMPLES,
                   "tile_variant": tile_variant,
                   "tile_variant_choice": "forced" if args.tile_variant >= 0 else "autotuned (timed once per batch)",
                   "selector": os.path.relpath(SELECTOR_MODEL, ROOT),
                   "l2": f"inputs larger than L2 ({in_bytes / 1e9:.1f} GB of A and B per batch), no flush"},
        "accuracy": stats,
        "selector_eval": sel_eval,
        "grouped_ms_without_graph": grouped_ms_nograph,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "compare": compare,
        "single_dgemm": single,
        "zgemm_kkr": zgemm,
        "regions": regions,
        "blas_shim_strategies": shim,
        "gpu_launches": launches,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


def main():
    global SELECTOR_MODEL
    args = parse()
    SELECTOR_MODEL = args.selector
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
