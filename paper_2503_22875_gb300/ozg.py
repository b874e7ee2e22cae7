"""Thin ctypes binding to the CUDA library libozg.so (include/ozg.h).

Argument marshalling only: every step of the emulated GEMM runs in the library's kernels.
PyTorch is used for device memory and streams (tensors are passed by ``data_ptr()``).
There is no CPU fallback: if the library is missing the import of this binding fails.

Matrices follow BLAS conventions (column-major).  A column-major m x n matrix with leading
dimension m has the same bytes as a row-major torch tensor of shape (n, m); the helpers
``to_device`` / ``from_device`` convert numpy arrays to and from that layout.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
SELECTOR_PARAMS = 6475


class OzgError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = f"{what} failed with code {code}: {strerror(code)}"
        if code == 1:
            msg += f" ({last_cuda_error()})"
        super().__init__(msg)


class GemmDesc(ctypes.Structure):
    """ozg_gemm_desc of include/ozg.h."""
    _fields_ = [("transa", ctypes.c_char), ("transb", ctypes.c_char), ("reserved", ctypes.c_char * 6),
                ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64)]


class Report(ctypes.Structure):
    _fields_ = [("slices_used", ctypes.c_int), ("nonfinite", ctypes.c_int), ("status", ctypes.c_int),
                ("samples", ctypes.c_int), ("est_err", ctypes.c_double), ("selected", ctypes.c_int),
                ("repaired", ctypes.c_int), ("max_real", ctypes.c_double), ("max_imag", ctypes.c_double)]


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libozg.so (built by ``__graft_entry__.build()`` / ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} is missing (run paper_2503_22875_gb300.build.build())")
    L = ctypes.CDLL(path)
    i64, dbl, i32, ch, vp = ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_char, ctypes.c_void_p
    L.ozg_create.argtypes = [ctypes.POINTER(vp), ctypes.c_size_t]
    L.ozg_destroy.argtypes = [vp]
    L.ozg_set_stream.argtypes = [vp, vp]
    L.ozg_sync.argtypes = [vp]
    L.ozg_strerror.argtypes = [i32]
    L.ozg_strerror.restype = ctypes.c_char_p
    L.ozg_last_cuda_error.restype = ctypes.c_char_p
    L.ozg_dgemm.argtypes = [vp, ch, ch, i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, i32, vp]
    L.ozg_zgemm.argtypes = [vp, ch, ch, i64, i64, i64, vp, vp, i64, vp, i64, vp, vp, i64, i32, vp]
    L.ozg_native_dgemm.argtypes = [vp, ch, ch, i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64]
    L.ozg_native_zgemm.argtypes = [vp, ch, ch, i64, i64, i64, vp, vp, i64, vp, i64, vp, vp, i64]
    L.ozg_debug_split.argtypes = [vp, ch, i64, i64, vp, i64, i32, vp, vp]
    L.ozg_debug_zsplit.argtypes = [vp, ch, i64, i64, vp, i64, i32, vp, vp]
    L.ozg_set_profiling.argtypes = [vp, i32]
    L.ozg_set_check_samples.argtypes = [vp, i32]
    L.ozg_set_exact_epilogue.argtypes = [vp, i32]
    L.ozg_phase_times.argtypes = [vp, vp, vp]
    L.ozg_dgemm_noalloc.argtypes = [ch, ch, i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, i32, vp]
    L.ozg_dgemm_grouped.argtypes = [vp, i64, vp, vp, vp]
    L.ozg_dgemm_grouped_host.argtypes = [vp, i64, vp, vp, vp]
    L.ozg_set_host_parts.argtypes = [vp, i32]
    L.ozg_zgemm3m.argtypes = [vp, ch, ch, i64, i64, i64, vp, vp, i64, vp, i64, vp, vp, i64, i32, vp]
    L.ozg_debug_wait.argtypes = [vp, ctypes.c_longlong]
    L.ozg_debug_fail_allocs.argtypes = [vp, i32]
    L.ozg_dgemm_regions.argtypes = [vp, ch, ch, i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, i32, i32, vp]
    L.ozg_load_selector.argtypes = [vp, ctypes.c_char_p]
    L.ozg_set_target_error.argtypes = [vp, dbl]
    L.ozg_selector_features.argtypes = [vp, ch, ch, i64, i64, i64, vp, i64, vp, i64, vp, vp, vp]
    L.ozg_selector_set_params.argtypes = [vp, vp]
    L.ozg_selector_get_params.argtypes = [vp, vp]
    L.ozg_selector_grads.argtypes = [vp, vp, vp, i32, vp, vp]
    L.ozg_selector_train_step.argtypes = [vp, vp, vp, i32, ctypes.c_float, vp]
    L.ozg_set_graphs.argtypes = [vp, i32]
    L.ozg_set_fallback_slices.argtypes = [vp, i32]
    L.ozg_set_autotune.argtypes = [vp, i32, ctypes.c_char_p]
    L.ozg_set_tile_variant.argtypes = [vp, i32]
    L.ozg_get_tile_variant.argtypes = [vp, ctypes.POINTER(i32)]
    L.ozg_kernel_launches.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
    L.ozg_debug_group_products.argtypes = [vp, ch, ch, i64, i64, i64, vp, i64, vp, i64, i32, vp]
    _lib = L
    return L


def kernel_launches() -> int:
    """Kernel launches the library has issued in this process (graph replays included)."""
    n = ctypes.c_longlong(0)
    _check(load().ozg_kernel_launches(ctypes.byref(n)), "ozg_kernel_launches")
    return int(n.value)


def strerror(code: int) -> str:
    return load().ozg_strerror(int(code)).decode()


def last_cuda_error() -> str:
    return load().ozg_last_cuda_error().decode()


def _p(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _hp(x) -> int:
    """Address of a host buffer: an int, a CPU torch tensor or a numpy array."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    return int(x.data_ptr())


def _c(t: str) -> bytes:
    return t.encode()


def _check(rc: int, what: str) -> int:
    if rc != 0:
        raise OzgError(rc, what)
    return rc


class Context:
    """An ozg_ctx: owns device workspace and queues work on one CUDA stream."""

    def __init__(self, workspace_bytes: int = 0, stream=None):
        L = load()
        h = ctypes.c_void_p()
        _check(L.ozg_create(ctypes.byref(h), int(workspace_bytes)), "ozg_create")
        self._h = h
        if stream is not None:
            self.set_stream(stream)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load().ozg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t (int) or None (legacy default)."""
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
        _check(load().ozg_set_stream(self._h, ctypes.c_void_p(raw)), "ozg_set_stream")

    def sync(self):
        _check(load().ozg_sync(self._h), "ozg_sync")

    PHASES = ("split", "gemm", "native", "check", "select", "grouped")

    def set_exact_epilogue(self, enable: bool):
        _check(load().ozg_set_exact_epilogue(self._h, int(bool(enable))), "ozg_set_exact_epilogue")

    def set_check_samples(self, samples: int):
        _check(load().ozg_set_check_samples(self._h, int(samples)), "ozg_set_check_samples")

    def set_profiling(self, enable: bool = True):
        _check(load().ozg_set_profiling(self._h, int(bool(enable))), "ozg_set_profiling")

    def phase_times(self):
        """{phase: (device ms, launches)} accumulated since the previous call (synchronises)."""
        ms = (ctypes.c_double * 8)()
        n = (ctypes.c_int64 * 8)()
        _check(load().ozg_phase_times(self._h, ms, n), "ozg_phase_times")
        return {name: (ms[i], n[i]) for i, name in enumerate(self.PHASES)}

    def dgemm(self, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices, report=False):
        rep = Report() if report else None
        rc = load().ozg_dgemm(self._h, _c(transa), _c(transb), m, n, k, float(alpha), _p(A), lda, _p(B), ldb,
                              float(beta), _p(C), ldc, int(slices), ctypes.byref(rep) if rep else None)
        _check(rc, "ozg_dgemm")
        return rep

    def zgemm(self, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices, report=False):
        rep = Report() if report else None
        al = (ctypes.c_double * 2)(complex(alpha).real, complex(alpha).imag)
        be = (ctypes.c_double * 2)(complex(beta).real, complex(beta).imag)
        rc = load().ozg_zgemm(self._h, _c(transa), _c(transb), m, n, k, al, _p(A), lda, _p(B), ldb, be, _p(C), ldc,
                              int(slices), ctypes.byref(rep) if rep else None)
        _check(rc, "ozg_zgemm")
        return rep

    def zgemm3m(self, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices, report=False):
        """3M complex product from three real emulated products (ozg_zgemm3m)."""
        rep = Report() if report else None
        al = (ctypes.c_double * 2)(complex(alpha).real, complex(alpha).imag)
        be = (ctypes.c_double * 2)(complex(beta).real, complex(beta).imag)
        rc = load().ozg_zgemm3m(self._h, _c(transa), _c(transb), m, n, k, al, _p(A), lda, _p(B), ldb, be, _p(C), ldc,
                                int(slices), ctypes.byref(rep) if rep else None)
        _check(rc, "ozg_zgemm3m")
        return rep

    def dgemm_grouped(self, calls, slices=None, report=False):
        """calls: sequence of (transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc) with
        device tensors or raw pointers; slices: per-call slice counts (0: the selector's choice when
        one is loaded, else the fallback count).  Returns the
        list of Report when report=True."""
        n = len(calls)
        arr = (GemmDesc * n)()
        for i, c in enumerate(calls):
            ta, tb, m, nn, k, al, A, lda, B, ldb, be, C, ldc = c
            arr[i] = GemmDesc(ta.encode(), tb.encode(), b"", m, nn, k, float(al), float(be), _p(A), lda, _p(B), ldb,
                              _p(C), ldc)
        sl = (ctypes.c_int * n)(*([0] * n if slices is None else [int(x) for x in slices]))
        reps = (Report * n)() if report else None
        rc = load().ozg_dgemm_grouped(self._h, n, arr, sl, reps)
        _check(rc, "ozg_dgemm_grouped")
        return list(reps) if report else None

    def dgemm_grouped_host(self, calls, slices=None, report=False):
        """ozg_dgemm_grouped_host: like dgemm_grouped, but A, B and C are host memory (raw
        addresses as ints, or CPU tensors / numpy arrays, passed by address).  Synchronous."""
        n = len(calls)
        arr = (GemmDesc * n)()
        for i, c in enumerate(calls):
            ta, tb, m, nn, k, al, A, lda, B, ldb, be, C, ldc = c
            arr[i] = GemmDesc(ta.encode(), tb.encode(), b"", m, nn, k, float(al), float(be), _hp(A), lda, _hp(B), ldb,
                              _hp(C), ldc)
        sl = (ctypes.c_int * n)(*([0] * n if slices is None else [int(x) for x in slices]))
        reps = (Report * n)() if report else None
        _check(load().ozg_dgemm_grouped_host(self._h, n, arr, sl, reps), "ozg_dgemm_grouped_host")
        return list(reps) if report else None

    def set_host_parts(self, parts: int):
        _check(load().ozg_set_host_parts(self._h, int(parts)), "ozg_set_host_parts")

    def dgemm_regions(self, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, row_blocks, col_blocks,
                      report=False):
        """C = alpha op(A) op(B) + beta C as row_blocks x col_blocks regions, each with the slice
        count the selector picks for it (one grouped launch).  Returns the band-row-major list of
        Report when report=True."""
        nreg = int(row_blocks) * int(col_blocks)
        reps = (Report * max(nreg, 1))() if report else None
        rc = load().ozg_dgemm_regions(self._h, _c(transa), _c(transb), m, n, k, float(alpha), _p(A), lda, _p(B), ldb,
                                      float(beta), _p(C), ldc, int(row_blocks), int(col_blocks), reps)
        _check(rc, "ozg_dgemm_regions")
        return list(reps)[:nreg] if report else None

    def set_graphs(self, enable: bool):
        _check(load().ozg_set_graphs(self._h, int(bool(enable))), "ozg_set_graphs")

    def set_fallback_slices(self, s: int):
        _check(load().ozg_set_fallback_slices(self._h, int(s)), "ozg_set_fallback_slices")

    def set_autotune(self, enable: bool, cache_path: str | None = None):
        _check(load().ozg_set_autotune(self._h, int(bool(enable)), cache_path.encode() if cache_path else None),
               "ozg_set_autotune")

    def set_tile_variant(self, variant: int):
        """Force tile variant 0..3 (bit 0: 128-wide tiles, bit 1: deferred epilogue pushes), or -1
        for the autotuned / heuristic choice."""
        _check(load().ozg_set_tile_variant(self._h, int(variant)), "ozg_set_tile_variant")

    def tile_variant(self) -> int:
        """Tile variant of the most recent grouped call (-1: none yet)."""
        v = ctypes.c_int(-1)
        _check(load().ozg_get_tile_variant(self._h, ctypes.byref(v)), "ozg_get_tile_variant")
        return int(v.value)

    # ---- learned slice selector
    def load_selector(self, path: str):
        _check(load().ozg_load_selector(self._h, path.encode()), "ozg_load_selector")

    def set_target_error(self, target: float):
        _check(load().ozg_set_target_error(self._h, float(target)), "ozg_set_target_error")

    def selector_features(self, transa, transb, m, n, k, A, lda, B, ldb, feat_out, prob_out=None, s_out=None):
        _check(load().ozg_selector_features(self._h, _c(transa), _c(transb), m, n, k, _p(A), lda, _p(B), ldb,
                                            _p(feat_out), _p(prob_out), _p(s_out)), "ozg_selector_features")

    def selector_set_params(self, theta: np.ndarray):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        _check(load().ozg_selector_set_params(self._h, t.ctypes.data), "ozg_selector_set_params")

    def selector_get_params(self) -> np.ndarray:
        t = np.zeros(SELECTOR_PARAMS, dtype=np.float32)
        _check(load().ozg_selector_get_params(self._h, t.ctypes.data), "ozg_selector_get_params")
        return t

    def selector_grads(self, X, y, B):
        g = np.zeros(SELECTOR_PARAMS, dtype=np.float32)
        loss = ctypes.c_float()
        _check(load().ozg_selector_grads(self._h, _p(X), _p(y), int(B), g.ctypes.data, ctypes.byref(loss)),
               "ozg_selector_grads")
        return float(loss.value), g

    def selector_train_step(self, X, y, B, lr):
        loss = ctypes.c_float()
        _check(load().ozg_selector_train_step(self._h, _p(X), _p(y), int(B), float(lr), ctypes.byref(loss)),
               "ozg_selector_train_step")
        return float(loss.value)

    def native_dgemm(self, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc):
        _check(load().ozg_native_dgemm(self._h, _c(transa), _c(transb), m, n, k, float(alpha), _p(A), lda, _p(B),
                                       ldb, float(beta), _p(C), ldc), "ozg_native_dgemm")

    def native_zgemm(self, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc):
        al = (ctypes.c_double * 2)(complex(alpha).real, complex(alpha).imag)
        be = (ctypes.c_double * 2)(complex(beta).real, complex(beta).imag)
        _check(load().ozg_native_zgemm(self._h, _c(transa), _c(transb), m, n, k, al, _p(A), lda, _p(B), ldb, be,
                                       _p(C), ldc), "ozg_native_zgemm")

    def debug_split(self, trans, rows, k, X, ld, slices, e_out, digits_out, complex_=False):
        f = load().ozg_debug_zsplit if complex_ else load().ozg_debug_split
        _check(f(self._h, _c(trans), rows, k, _p(X), ld, int(slices), _p(e_out), _p(digits_out)), "ozg_debug_split")

    def debug_group_products(self, transa, transb, m, n, k, A, lda, B, ldb, slices, G_out):
        _check(load().ozg_debug_group_products(self._h, _c(transa), _c(transb), m, n, k, _p(A), lda, _p(B), ldb,
                                               int(slices), _p(G_out)), "ozg_debug_group_products")


def dgemm_noalloc(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices, stream=None) -> int:
    """ozg_dgemm_noalloc: the emulated DGEMM with no device allocation (fixed in-library scratch),
    for callers that cannot call cudaMalloc.  Returns the library's return code unchanged."""
    raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
    return int(load().ozg_dgemm_noalloc(_c(transa), _c(transb), m, n, k, float(alpha), _p(A), lda, _p(B), ldb,
                                        float(beta), _p(C), ldc, int(slices), ctypes.c_void_p(raw)))


# ------------------------------------------------------------------- layout helpers (marshalling)
def to_device(x: np.ndarray, device="cuda"):
    """numpy (m, n) -> torch tensor holding the column-major bytes of x (shape (n, m))."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asfortranarray(x).T)).to(device)


def from_device(t, m: int, n: int) -> np.ndarray:
    """Inverse of to_device for an m x n column-major matrix stored in t."""
    a = t.detach().cpu().numpy().reshape(n, m)
    return np.asfortranarray(a.T)
