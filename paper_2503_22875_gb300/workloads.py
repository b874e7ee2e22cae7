"""Seeded synthetic inputs shaped like the workloads of the paper's study (Sec. 3.2 / 4).

This module holds no arithmetic of the emulation method: it only draws random matrices, so it
can feed both the CUDA path and the CPU oracle.  numpy PCG64 generators with fixed seeds.

  uniform_pair          A, B ~ U(-1, 1)                         (small DGEMM, m = n = k = 256)
  wide_exponent_pair    a = (u - 0.5) exp(phi g), u ~ U(0,1), g ~ N(0,1)   (8192^3 DGEMM sweep)
  kkr_like_pair         complex n = 113 blocks x 32, block (i,j) ~ CN(0,1) exp(-|r_i - r_j|)
                        with atom sites r ~ U(cube of unit density) plus (1 + 0.1i) on the
                        diagonal -- stands in for the MuST "MT u56" ZGEMMs of Sec. 3.2
  kkr_kappa_pair        the same with A's diagonal shift moved next to an eigenvalue of the
                        unshifted matrix so that cond_2(A) ~ 1e8 (shift found once, cached)
  grouped_batch         2048 GEMMs, m, n, k log-uniform in [32, 2048], phi ~ U(0, 4) per call
                        (grouped_batch_flat: the same batch drawn on the GPU into flat buffers)
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_pair(m: int, n: int, k: int, seed: int = 1):
    g = rng(seed)
    A = np.asfortranarray(g.uniform(-1.0, 1.0, size=(m, k)))
    B = np.asfortranarray(g.uniform(-1.0, 1.0, size=(k, n)))
    return A, B


def wide_exponent(shape, phi: float, g: np.random.Generator) -> np.ndarray:
    u = g.random(size=shape)
    z = g.standard_normal(size=shape)
    return np.asfortranarray((u - 0.5) * np.exp(phi * z))


def wide_exponent_pair(m: int, n: int, k: int, phi: float, seed: int = 2):
    g = rng(seed)
    return wide_exponent((m, k), phi, g), wide_exponent((k, n), phi, g)


def _kkr_matrix(nblk: int, bs: int, g: np.random.Generator, shift: complex) -> np.ndarray:
    L = nblk ** (1.0 / 3.0)
    r = g.uniform(0.0, L, size=(nblk, 3))
    d = np.sqrt(((r[:, None, :] - r[None, :, :]) ** 2).sum(-1))
    scale = np.exp(-d)  # (nblk, nblk)
    n = nblk * bs
    M = (g.standard_normal(size=(n, n)) + 1j * g.standard_normal(size=(n, n))) / np.sqrt(2.0)
    M *= np.repeat(np.repeat(scale, bs, axis=0), bs, axis=1)
    M[np.arange(n), np.arange(n)] += shift
    return np.asfortranarray(M)


def kkr_like_pair(nblk: int = 113, bs: int = 32, seed: int = 3, shift: complex = 1.0 + 0.1j):
    """Two independently seeded KKR-like complex matrices of order nblk * bs."""
    g = rng(seed)
    A = _kkr_matrix(nblk, bs, g, shift)
    B = _kkr_matrix(nblk, bs, g, shift)
    return A, B


KAPPA_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "kkr_kappa_shift.json")


def _cond2(M) -> float:
    sv = np.linalg.svd(M, compute_uv=False)
    return float(sv[0] / sv[-1])


def kkr_kappa_shift(nblk: int = 113, bs: int = 32, seed: int = 3, kappa: float = 1e8, cache: str = KAPPA_CACHE,
                    log=None) -> complex:
    """Diagonal shift of A (the first matrix of kkr_like_pair) for which cond_2(A) is within a
    factor 1.5 of `kappa`: shift = -lambda + t u, with lambda the eigenvalue of the unshifted
    matrix M nearest to -(1 + 0.1i) and u the unit direction from -lambda towards 1 + 0.1i;
    t by bisection on log t (cond_2 grows without bound as t -> 0).  Computed once per
    (nblk, bs, seed, kappa) with LAPACK on the host and cached as JSON."""
    key = f"{nblk}x{bs}:seed{seed}:kappa{kappa:g}"
    table = {}
    if os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
    if key in table:
        return complex(table[key]["re"], table[key]["im"])
    g = rng(seed)
    M = _kkr_matrix(nblk, bs, g, 0.0)
    lam = np.linalg.eigvals(M)
    base = -(1.0 + 0.1j)
    l0 = lam[np.argmin(np.abs(lam - base))]
    u = ((1.0 + 0.1j) - (-l0)) / abs((1.0 + 0.1j) - (-l0))
    n = M.shape[0]
    idx = np.arange(n)

    def cond_at(t):
        A = M.copy()
        A[idx, idx] += -l0 + t * u
        return _cond2(A)
    lo, hi = 1e-12, abs((1.0 + 0.1j) + l0)  # cond(lo) >> kappa, cond(hi) = the base matrix's
    for _ in range(40):
        mid = np.sqrt(lo * hi)
        c = cond_at(mid)
        if log:
            log(f"  t = {mid:.3e}: cond_2 = {c:.3e}")
        if c > kappa:
            lo = mid
        else:
            hi = mid
        if kappa / 1.5 <= c <= kappa * 1.5:
            break
    shift = complex(-l0 + mid * u)
    table[key] = {"re": shift.real, "im": shift.imag, "cond2": c, "t": mid}
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    with open(cache, "w") as f:
        json.dump(table, f, indent=1)
    return shift


def kkr_kappa_pair(nblk: int = 113, bs: int = 32, seed: int = 3, kappa: float = 1e8):
    """kkr_like_pair with A's diagonal shift replaced so that cond_2(A) ~ kappa."""
    g = rng(seed)
    M = _kkr_matrix(nblk, bs, g, 0.0)
    B = _kkr_matrix(nblk, bs, g, 1.0 + 0.1j)
    n = M.shape[0]
    M[np.arange(n), np.arange(n)] += kkr_kappa_shift(nblk, bs, seed, kappa)
    return np.asfortranarray(M), B


@dataclass
class GemmCall:
    m: int
    n: int
    k: int
    phi: float
    seed: int


def grouped_batch(count: int = 2048, lo: int = 32, hi: int = 2048, phi_hi: float = 4.0, seed: int = 4):
    """Shapes and per-call exponent spreads of the grouped batch; matrices via call_matrices()."""
    g = rng(seed)
    dims = np.exp(g.uniform(np.log(lo), np.log(hi), size=(count, 3))).round().astype(int)
    phis = g.uniform(0.0, phi_hi, size=count)
    seeds = g.integers(0, 2 ** 31 - 1, size=count)
    return [GemmCall(int(d[0]), int(d[1]), int(d[2]), float(p), int(s)) for d, p, s in zip(dims, phis, seeds)]


def call_matrices(c: GemmCall):
    return wide_exponent_pair(c.m, c.n, c.k, c.phi, seed=c.seed)


def grouped_batch_device(count: int = 2048, lo: int = 32, hi: int = 2048, phi_hi: float = 4.0, seed: int = 4,
                         device: str = "cuda"):
    """The grouped batch drawn directly on the GPU (torch generator, seeded): the same shape and
    spread distribution as grouped_batch, for benchmark-sized batches.  Returns a list of
    (m, n, k, phi, A, B) with A (m x k) and B (k x n) as column-major torch tensors."""
    import torch
    calls = grouped_batch(count, lo, hi, phi_hi, seed)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    out = []
    for c in calls:
        def draw(rows, cols):
            u = torch.rand((cols, rows), generator=gen, device=device, dtype=torch.float64)
            z = torch.randn((cols, rows), generator=gen, device=device, dtype=torch.float64)
            return (u - 0.5) * torch.exp(c.phi * z)  # shape (cols, rows): column-major rows x cols
        out.append((c.m, c.n, c.k, c.phi, draw(c.m, c.k), draw(c.k, c.n)))
    return out


@dataclass
class FlatBatch:
    """A grouped batch in three flat device buffers (A's, B's, C's back to back, 256-byte aligned
    offsets), so the whole batch moves between host and device in three copies."""
    calls: list          # GemmCall per problem
    A: object            # torch float64 flat buffers on the device
    B: object
    C: object
    offA: list           # element offsets of each problem's A, B, C
    offB: list
    offC: list

    def views(self, i):
        """(A_i, B_i, C_i) as column-major torch views: shapes (k, m), (n, k), (n, m)."""
        c = self.calls[i]
        a = self.A[self.offA[i]:self.offA[i] + c.m * c.k].view(c.k, c.m)
        b = self.B[self.offB[i]:self.offB[i] + c.k * c.n].view(c.n, c.k)
        cc = self.C[self.offC[i]:self.offC[i] + c.m * c.n].view(c.n, c.m)
        return a, b, cc

    def gemm_calls(self, alpha=1.0, beta=0.0):
        """Descriptor tuples ('N', 'N', m, n, k, alpha, A, lda, B, ldb, beta, C, ldc) for ozg."""
        out = []
        for i, c in enumerate(self.calls):
            a, b, cc = self.views(i)
            out.append(("N", "N", c.m, c.n, c.k, alpha, a, c.m, b, c.k, beta, cc, c.m))
        return out


def grouped_batch_flat(count: int = 2048, lo: int = 32, hi: int = 2048, phi_hi: float = 4.0, seed: int = 4,
                       device: str = "cuda") -> FlatBatch:
    """The grouped batch (shapes and spreads of grouped_batch) drawn on the GPU into flat buffers
    with a seeded torch generator."""
    import torch
    calls = grouped_batch(count, lo, hi, phi_hi, seed)

    def offsets(sizes):
        offs, o = [], 0
        for z in sizes:
            offs.append(o)
            o += (z + 31) // 32 * 32
        return offs, max(o, 1)

    offA, nA = offsets([c.m * c.k for c in calls])
    offB, nB = offsets([c.k * c.n for c in calls])
    offC, nC = offsets([c.m * c.n for c in calls])
    A = torch.zeros(nA, dtype=torch.float64, device=device)
    B = torch.zeros(nB, dtype=torch.float64, device=device)
    C = torch.zeros(nC, dtype=torch.float64, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    for i, c in enumerate(calls):
        for buf, off, size in ((A, offA[i], c.m * c.k), (B, offB[i], c.k * c.n)):
            u = torch.rand(size, generator=gen, device=device, dtype=torch.float64)
            z = torch.randn(size, generator=gen, device=device, dtype=torch.float64)
            buf[off:off + size] = (u - 0.5) * torch.exp(c.phi * z)
    return FlatBatch(calls, A, B, C, offA, offB, offC)
