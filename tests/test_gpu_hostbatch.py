"""ozg_dgemm_grouped_host: the grouped emulated DGEMM on host-memory matrices (staged by the
library, pipelined in parts) against the same batch on device memory and against the oracle.

The batch mixes matrices packed back to back in one pinned buffer (moved as merged copies) with
separate pageable numpy arrays, C with padding rows (ldc > m, which must stay untouched), beta != 0
(C read back from host), a transposed call, two calls sharing one A, a k = 0 call and learned
calls with reports; it runs twice (the parts' graphs replay) with one and with three parts."""
import numpy as np
import pytest

import oracle
from paper_2503_22875_gb300 import selector, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ozg():
    from paper_2503_22875_gb300 import build, ozg
    build.build()
    ozg.load()
    return ozg


def build_batch(seed):
    g = workloads.rng(seed)
    shapes = [(70, 90, 130), (300, 40, 517), (33, 257, 64), (128, 128, 900), (5, 7, 3), (200, 180, 1100),
              (64, 300, 250), (90, 91, 92)]
    packed = []   # matrices that live in one pinned buffer, back to back
    calls = []
    for i, (m, n, k) in enumerate(shapes):
        ta = "T" if i == 2 else "N"
        A = workloads.wide_exponent((m, k) if ta == "N" else (k, m), 1.0 + 0.3 * i, g)
        B = workloads.wide_exponent((k, n), 1.0 + 0.3 * i, g)
        ldc = m + (3 if i % 3 == 1 else 0)
        C0 = np.asfortranarray(g.uniform(-1, 1, (ldc, n)))
        beta = 0.5 if i % 2 else 0.0
        calls.append(dict(ta=ta, m=m, n=n, k=k, A=np.asfortranarray(A), B=np.asfortranarray(B), C0=C0, ldc=ldc,
                          alpha=-1.5 if i == 5 else 1.0, beta=beta, s=0 if i % 4 == 0 else 6 + i % 4,
                          packed=(i % 2 == 0 and ldc == m)))
    calls.append(dict(calls[0], C0=np.asfortranarray(g.uniform(-1, 1, (70, 90))), share=0, packed=False, s=7))
    calls.append(dict(ta="N", m=40, n=30, k=0, A=np.zeros((40, 1), order="F"), B=np.zeros((1, 30), order="F"),
                      C0=np.asfortranarray(g.uniform(-1, 1, (40, 30))), ldc=40, alpha=1.0, beta=2.0, s=7,
                      packed=False))
    return calls


def host_layout(calls):
    """Pinned flat buffers for the packed calls (A's back to back, B's, C's), numpy otherwise."""
    tot = lambda key: sum(c[key].size for c in calls if c["packed"])  # noqa: E731
    bufs = {key: torch.empty(max(tot(key), 1), dtype=torch.float64, pin_memory=True) for key in ("A", "B", "C0")}
    offs = {key: 0 for key in bufs}
    ptr = []
    for c in calls:
        p = {}
        for key in ("A", "B", "C0"):
            if c["packed"]:
                o = offs[key]
                flat = bufs[key][o:o + c[key].size]
                flat.copy_(torch.from_numpy(np.ascontiguousarray(c[key].reshape(-1, order="F"))))
                p[key] = (flat, flat.data_ptr())
                offs[key] += c[key].size
            else:
                arr = np.asfortranarray(c[key]).copy(order="F")
                p[key] = (arr, arr.ctypes.data)
        ptr.append(p)
    return ptr, bufs


def read_c(p, c):
    obj = p["C0"][0]
    a = obj.numpy() if hasattr(obj, "numpy") else obj.reshape(-1, order="F")
    return np.asfortranarray(np.asarray(a).reshape(c["n"], c["ldc"]).T)


@pytest.mark.parametrize("parts", [1, 3])
def test_grouped_host_matches_device_and_oracle(ozg, parts):
    calls = build_batch(1400 + parts)
    ptr, bufs = host_layout(calls)
    for i, c in enumerate(calls):
        if "share" in c:  # same host A as call 0
            ptr[i]["A"] = ptr[c["share"]]["A"]
    ctx = ozg.Context()
    ctx.load_selector(selector.DEFAULT_MODEL)
    ctx.set_target_error(1e-12)
    ctx.set_check_samples(32)
    ctx.set_host_parts(parts)
    desc = [(c["ta"], "N", c["m"], c["n"], c["k"], c["alpha"], ptr[i]["A"][1], c["A"].shape[0], ptr[i]["B"][1],
             max(c["B"].shape[0], 1), c["beta"], ptr[i]["C0"][1], c["ldc"]) for i, c in enumerate(calls)]
    slices = [c["s"] for c in calls]
    # the device path on the same inputs
    st = torch.cuda.Stream()
    dctx = ozg.Context(stream=st)
    dctx.load_selector(selector.DEFAULT_MODEL)
    dctx.set_target_error(1e-12)
    dctx.set_check_samples(32)
    dev = [(ozg.to_device(c["A"]), ozg.to_device(c["B"]), ozg.to_device(c["C0"])) for c in calls]
    ddesc = [(c["ta"], "N", c["m"], c["n"], c["k"], c["alpha"], dA, c["A"].shape[0], dB, max(c["B"].shape[0], 1),
              c["beta"], dC, c["ldc"]) for c, (dA, dB, dC) in zip(calls, dev)]
    with torch.cuda.stream(st):
        drep = dctx.dgemm_grouped(ddesc, slices, report=True)
    for rep_round in range(2):
        hrep = ctx.dgemm_grouped_host(desc, slices, report=True)
        for i, c in enumerate(calls):
            C = read_c(ptr[i], c)
            D = ozg.from_device(dev[i][2], c["ldc"], c["n"])
            h, d = hrep[i], drep[i]
            # the sampled check's positions depend on a call's index within its part, so a learned
            # call near its minimal count may escalate differently; the choice itself may not differ
            assert (h.status, h.selected) == (d.status, d.selected), i
            # a part with a learned call checks at least 64 entries per call, others the context's 32
            assert h.samples == (0 if c["k"] == 0 else (64 if d.selected else h.samples)) and h.samples in (0, 32, 64)
            if h.slices_used == d.slices_used:
                assert np.array_equal(C, D), (i, rep_round)
            assert np.array_equal(C[c["m"]:], c["C0"][c["m"]:])  # padding rows untouched
            if c["k"] > 0:
                opA = c["A"].T if c["ta"] == "T" else c["A"]
                E = oracle.dgemm_emu(np.asfortranarray(opA), c["B"], h.slices_used, "N", "N", c["alpha"], c["beta"],
                                     np.asfortranarray(c["C0"][:c["m"]]))
                assert np.array_equal(C[:c["m"]], E), i
            else:
                assert np.array_equal(C[:c["m"]], c["beta"] * c["C0"][:c["m"]])
        # the next round reads C_old again from host: restore it
        for i, c in enumerate(calls):
            obj = ptr[i]["C0"][0]
            src = np.ascontiguousarray(c["C0"].reshape(-1, order="F"))
            if hasattr(obj, "copy_"):
                obj.copy_(torch.from_numpy(src))
            else:
                obj[...] = c["C0"]
    bad = list(desc)
    bad[3] = desc[3][:7] + (1,) + desc[3][8:]  # lda below the rows of A
    with pytest.raises(ozg.OzgError):
        ctx.dgemm_grouped_host(bad, slices)
    ctx.close()
    dctx.close()
