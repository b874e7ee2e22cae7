"""CPU oracle for Ozaki-scheme FP64 / complex128 GEMM emulation with INT8-range slices.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously-correct CPU reference
that the CUDA library is checked against (Sec. 2.2 of the paper: the Ozaki scheme on an
integer matrix-multiply unit, with the split number as the tunable precision of Sec. 3.1).
It shares no code with the CUDA path and must never be called by it: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it.

The arithmetic lives in ``ozaki_oracle.c`` (plain C, FP64, double-double and exact
multi-limb integers), compiled on first use with gcc.  Every function here is a thin
ctypes marshaller plus, where noted, a tiny pure-Python definition used for pinning.

Parity status: every function below is pinned by ``tests/test_oracle_*.py`` against exact
rational arithmetic, brute force on tiny inputs, closed forms or invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ozaki_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_CFLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11", "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    """Compile ozaki_oracle.c into _build/liboracle.so (gcc); returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *_CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # OZG_ORACLE_LIB: a separately compiled copy of this file's C source (the mutation
            # tests load copies with one planted mistake each and expect the pins to fail)
            lib = ctypes.CDLL(os.environ.get("OZG_ORACLE_LIB") or build())
            c_i64, c_dbl, c_int, c_char, vp = (ctypes.c_int64, ctypes.c_double, ctypes.c_int,
                                               ctypes.c_char, ctypes.c_void_p)
            lib.orc_dgemm_naive.argtypes = [c_char, c_char, c_i64, c_i64, c_i64, c_dbl, vp, c_i64, vp, c_i64,
                                            c_dbl, vp, c_i64]
            lib.orc_dgemm_dd.argtypes = [c_char, c_char, c_i64, c_i64, c_i64, c_dbl, vp, c_i64, vp, c_i64,
                                         c_dbl, vp, c_i64, vp, vp]
            lib.orc_zgemm_dd.argtypes = [c_char, c_char, c_i64, c_i64, c_i64, vp, c_i64, vp, c_i64, vp, vp, vp, vp]
            lib.orc_zgemm_naive.argtypes = [c_char, c_char, c_i64, c_i64, c_i64, vp, vp, c_i64, vp, c_i64,
                                            vp, vp, c_i64]
            lib.orc_split.argtypes = [c_char, c_i64, c_i64, vp, c_i64, c_int, vp, vp]
            lib.orc_zsplit.argtypes = [c_char, c_i64, c_i64, vp, c_i64, c_int, vp, vp]
            lib.orc_group_products.argtypes = [c_i64, c_i64, c_i64, c_int, vp, vp, c_int, vp]
            lib.orc_group_products.restype = c_int
            lib.orc_dgemm_emu.argtypes = [c_char, c_char, c_i64, c_i64, c_i64, c_dbl, vp, c_i64, vp, c_i64,
                                          c_dbl, vp, c_i64, c_int, c_int]
            lib.orc_zgemm_emu.argtypes = [c_char, c_char, c_i64, c_i64, c_i64, vp, vp, c_i64, vp, c_i64,
                                          vp, vp, c_i64, c_int]
            lib.orc_zgemm3m_combine.argtypes = [c_i64, c_i64, vp, vp, vp, vp, vp, vp, c_i64]
            lib.orc_emu_bound.argtypes = [c_char, c_char, c_i64, c_i64, c_i64, vp, c_i64, vp, c_i64, c_int, vp]
            lib.orc_mlp_loss_grad.argtypes = [vp, vp, vp, c_int, vp]
            lib.orc_mlp_loss_grad.restype = c_dbl
            lib.orc_mlp_select.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_float, c_int, c_int, vp, c_int, vp]
            lib.orc_mlp_select.restype = c_int
            lib.orc_features.argtypes = [c_char, c_char, c_i64, c_i64, c_i64, vp, c_i64, vp, c_i64, c_dbl, vp]
            lib.orc_bf16_round.argtypes = [ctypes.c_float]
            lib.orc_bf16_round.restype = ctypes.c_float
            lib.orc_set_threads.argtypes = [c_int]
            lib.orc_get_threads.restype = c_int
            _lib = lib
    return _lib


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def threads() -> int:
    return int(_load().orc_get_threads())


# ----------------------------------------------------------------------------- helpers
def _fortran(x: np.ndarray, dtype) -> np.ndarray:
    return np.asfortranarray(np.asarray(x, dtype=dtype))


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _op_shape(t: str, a: np.ndarray):
    return a.shape if t in "Nn" else (a.shape[1], a.shape[0])


def _b(t: str) -> bytes:
    return t.encode()


# ----------------------------------------------------------------------------- real GEMMs
def dgemm_naive(A, B, transa="N", transb="N", alpha=1.0, beta=0.0, C=None):
    """O-naive: C = alpha op(A) op(B) + beta C in plain FP64, k ascending (no FMA)."""
    A, B = _fortran(A, np.float64), _fortran(B, np.float64)
    m, k = _op_shape(transa, A)
    k2, n = _op_shape(transb, B)
    assert k == k2
    C = np.zeros((m, n), order="F") if C is None else np.array(C, dtype=np.float64, order="F", copy=True)
    _load().orc_dgemm_naive(_b(transa), _b(transb), m, n, k, float(alpha), _ptr(A), max(A.shape[0], 1),
                            _ptr(B), max(B.shape[0], 1), float(beta), _ptr(C), max(m, 1))
    return C


def dgemm_dd(A, B, transa="N", transb="N", alpha=1.0, beta=0.0, C=None):
    """O-dd: alpha op(A) op(B) + beta C in double-double; returns (hi, lo) arrays."""
    A, B = _fortran(A, np.float64), _fortran(B, np.float64)
    m, k = _op_shape(transa, A)
    k2, n = _op_shape(transb, B)
    assert k == k2
    Cw = np.zeros((m, n), order="F") if C is None else np.array(C, dtype=np.float64, order="F", copy=True)
    hi = np.zeros((m, n), order="F")
    lo = np.zeros((m, n), order="F")
    _load().orc_dgemm_dd(_b(transa), _b(transb), m, n, k, float(alpha), _ptr(A), max(A.shape[0], 1),
                         _ptr(B), max(B.shape[0], 1), float(beta), _ptr(Cw), max(m, 1), _ptr(hi), _ptr(lo))
    return hi, lo


def zgemm_dd(A, B, transa="N", transb="N"):
    """Complex double-double product op(A) op(B); returns (re_hi, re_lo, im_hi, im_lo)."""
    A, B = _fortran(A, np.complex128), _fortran(B, np.complex128)
    m, k = _op_shape(transa, A)
    k2, n = _op_shape(transb, B)
    assert k == k2
    outs = [np.zeros((m, n), order="F") for _ in range(4)]
    _load().orc_zgemm_dd(_b(transa), _b(transb), m, n, k, _ptr(A), max(A.shape[0], 1), _ptr(B),
                         max(B.shape[0], 1), *[_ptr(o) for o in outs])
    return tuple(outs)


def zgemm_naive(A, B, transa="N", transb="N", alpha=1.0, beta=0.0, C=None):
    A, B = _fortran(A, np.complex128), _fortran(B, np.complex128)
    m, k = _op_shape(transa, A)
    k2, n = _op_shape(transb, B)
    C = np.zeros((m, n), order="F", dtype=np.complex128) if C is None else np.array(C, dtype=np.complex128, order="F", copy=True)
    al = np.array([complex(alpha).real, complex(alpha).imag])
    be = np.array([complex(beta).real, complex(beta).imag])
    _load().orc_zgemm_naive(_b(transa), _b(transb), m, n, k, _ptr(al), _ptr(A), max(A.shape[0], 1),
                            _ptr(B), max(B.shape[0], 1), _ptr(be), _ptr(C), max(m, 1))
    return C


# ----------------------------------------------------------------------------- splitting
def split(X, s: int, trans: str = "N"):
    """O-slice for the rows of op(X): returns (e[rows] int32, D[s, rows, k] int8)."""
    X = _fortran(X, np.float64)
    rows, k = _op_shape(trans, X)
    e = np.zeros(rows, dtype=np.int32)
    D = np.zeros((s, rows, k), dtype=np.int8)
    _load().orc_split(_b(trans), rows, k, _ptr(X), max(X.shape[0], 1), int(s), _ptr(e), _ptr(D))
    return e, D


def split_cols(X, s: int, trans: str = "N"):
    """O-slice for the columns of op(X) (the B operand): (f[cols], D[s, cols, k])."""
    return split(X, s, "T" if trans in "Nn" else "N")


def zsplit(X, s: int, trans: str = "N"):
    """Complex O-slice of the rows of op(X): (e[rows], D[s, 2*rows, k]) with interleaved
    Re (row 2i) / Im (row 2i+1) digit rows sharing one exponent per complex row."""
    X = _fortran(X, np.complex128)
    rows, k = _op_shape(trans, X)
    e = np.zeros(rows, dtype=np.int32)
    D = np.zeros((s, 2 * rows, k), dtype=np.int8)
    _load().orc_zsplit(_b(trans), rows, k, _ptr(X), max(X.shape[0], 1), int(s), _ptr(e), _ptr(D))
    return e, D


def group_products(DA, DB, square: bool = False):
    """O-int: G[g-2] = sum_{p+q=g} DA[p-1] DB[q-1]^T exactly (int64)."""
    DA = np.ascontiguousarray(DA, dtype=np.int8)
    DB = np.ascontiguousarray(DB, dtype=np.int8)
    s, m, k = DA.shape
    s2, n, k2 = DB.shape
    assert s == s2 and k == k2
    ng = 2 * s - 1 if square else s
    G = np.zeros((ng, m, n), dtype=np.int64)
    _load().orc_group_products(m, n, k, s, _ptr(DA), _ptr(DB), int(bool(square)), _ptr(G))
    return G


# ----------------------------------------------------------------------------- emulation
def dgemm_emu(A, B, s: int, transa="N", transb="N", alpha=1.0, beta=0.0, C=None, square=False):
    """O-emu: C = alpha RN(T) + beta C_old with T from the exact slice products."""
    A, B = _fortran(A, np.float64), _fortran(B, np.float64)
    m, k = _op_shape(transa, A)
    k2, n = _op_shape(transb, B)
    assert k == k2
    C = np.zeros((m, n), order="F") if C is None else np.array(C, dtype=np.float64, order="F", copy=True)
    _load().orc_dgemm_emu(_b(transa), _b(transb), m, n, k, float(alpha), _ptr(A), max(A.shape[0], 1),
                          _ptr(B), max(B.shape[0], 1), float(beta), _ptr(C), max(m, 1), int(s),
                          int(bool(square)))
    return C


def zgemm_emu(A, B, s: int, transa="N", transb="N", alpha=1.0, beta=0.0, C=None):
    A, B = _fortran(A, np.complex128), _fortran(B, np.complex128)
    m, k = _op_shape(transa, A)
    k2, n = _op_shape(transb, B)
    assert k == k2
    C = np.zeros((m, n), order="F", dtype=np.complex128) if C is None else np.array(C, dtype=np.complex128, order="F", copy=True)
    al = np.array([complex(alpha).real, complex(alpha).imag])
    be = np.array([complex(beta).real, complex(beta).imag])
    _load().orc_zgemm_emu(_b(transa), _b(transb), m, n, k, _ptr(al), _ptr(A), max(A.shape[0], 1),
                          _ptr(B), max(B.shape[0], 1), _ptr(be), _ptr(C), max(m, 1), int(s))
    return C


def _op(X, t: str):
    """op(X) as a column-major array: X, X^T or X^H."""
    X = np.asarray(X)
    return np.asfortranarray(X if t in "Nn" else (X.T if t in "Tt" else X.conj().T))


def zgemm3m_operands(A, B, transa="N", transb="N"):
    """The real operands of the 3M product: (Ar, Ai, Sa) of op(A) and (Br, Bi, Sb) of op(B), with
    Sa = RN(Ar + Ai) and Sb = RN(Br + Bi) (one FP64 addition each), all column-major."""
    oA, oB = _op(np.asarray(A, dtype=np.complex128), transa), _op(np.asarray(B, dtype=np.complex128), transb)
    Ar, Ai = np.asfortranarray(oA.real), np.asfortranarray(oA.imag)
    Br, Bi = np.asfortranarray(oB.real), np.asfortranarray(oB.imag)
    return (Ar, Ai, np.asfortranarray(Ar + Ai)), (Br, Bi, np.asfortranarray(Br + Bi))


def zgemm3m_emu(A, B, s: int, transa="N", transb="N", alpha=1.0, beta=0.0, C=None):
    """O-emu 3M: complex C = alpha op(A) op(B) + beta C from THREE real emulated products (the
    Karatsuba form, 3 real products instead of 4): P1 = emu(Ar, Br), P2 = emu(Ai, Bi),
    P3 = emu(Sa, Sb); Re = RN(P1 - P2), Im = RN(RN(P3 - P1) - P2); alpha, beta as zgemm_emu.
    The paper builds complex products from real sub-products (Sec. 2.2, Sec. 3.2) but does not
    describe a 3M form; each real product here is dgemm_emu (Sec. 2.2's scheme)."""
    (Ar, Ai, Sa), (Br, Bi, Sb) = zgemm3m_operands(A, B, transa, transb)
    m, n = Ar.shape[0], Br.shape[1]
    P1, P2, P3 = dgemm_emu(Ar, Br, s), dgemm_emu(Ai, Bi, s), dgemm_emu(Sa, Sb, s)
    C = np.zeros((m, n), order="F", dtype=np.complex128) if C is None else np.array(C, dtype=np.complex128, order="F", copy=True)
    if m == 0 or n == 0:
        return C
    al = np.array([complex(alpha).real, complex(alpha).imag])
    be = np.array([complex(beta).real, complex(beta).imag])
    _load().orc_zgemm3m_combine(m, n, _ptr(P1), _ptr(P2), _ptr(P3), _ptr(al), _ptr(be), _ptr(C), max(m, 1))
    return C


def zgemm3m_bound(A, B, s: int, transa="N", transb="N"):
    """O-bound 3M: a priori |Re(T) - Re(op(A)op(B))| and |Im(T) - Im(op(A)op(B))| per entry of the
    3M result T (alpha = 1, beta = 0).  With e(X, Y) = emu_bound(X, Y) (the exact-arithmetic
    emulation error), |P - XY| <= e(X, Y) + u |P| for each rounded product, and
    |Sa Sb - (Ar + Ai)(Br + Bi)| <= (2u + u^2) (|Ar| + |Ai|)(|Br| + |Bi|).  The real part adds
    one rounding of P1 - P2, the imaginary part two:
      re: e1 + e2 + u(|P1| + |P2|) + u |t_r|
      im: e3 + e1 + e2 + u(|P3| + |P1| + |P2|) + (2u + u^2)(|Ar| + |Ai|)(|Br| + |Bi|)
          + u |P3 - P1| + u |t_i|
    with |P| <= ((|X||Y|)(1 + 2(k + 1)u) + e)(1 + u): the FP64 evaluation of |X||Y| is within
    gamma_k of the exact one, so no result is needed to evaluate the bound."""
    (Ar, Ai, Sa), (Br, Bi, Sb) = zgemm3m_operands(A, B, transa, transb)
    u = 2.0 ** -53
    k = Ar.shape[1]
    g = 1 + 2 * (k + 2) * u
    e1, e2, e3 = emu_bound(Ar, Br, s), emu_bound(Ai, Bi, s), emu_bound(Sa, Sb, s)
    a1, a2, a3 = abs_product(Ar, Br), abs_product(Ai, Bi), abs_product(Sa, Sb)
    q = abs_product(np.abs(Ar) + np.abs(Ai), np.abs(Br) + np.abs(Bi)) * g
    P1, P2, P3 = ((a * g + e) * (1 + u) for a, e in ((a1, e1), (a2, e2), (a3, e3)))
    re = e1 + e2 + u * (P1 + P2) + u * (P1 + P2) * (1 + u)
    d = (P3 + P1) * (1 + u)
    im = e3 + e1 + e2 + u * (P3 + P1 + P2) + (2 * u + u * u) * q + u * d + u * (d + P2) * (1 + u)
    return re * (1 + 16 * u), im * (1 + 16 * u)


def emu_bound(A, B, s: int, transa="N", transb="N"):
    """O-bound: a priori |op(A)op(B) - T| per entry (final rounding not included)."""
    A, B = _fortran(A, np.float64), _fortran(B, np.float64)
    m, k = _op_shape(transa, A)
    k2, n = _op_shape(transb, B)
    out = np.zeros((m, n), order="F")
    _load().orc_emu_bound(_b(transa), _b(transb), m, n, k, _ptr(A), max(A.shape[0], 1), _ptr(B),
                          max(B.shape[0], 1), int(s), _ptr(out))
    return out


def abs_product(A, B, transa="N", transb="N"):
    """(|op(A)| |op(B)|) in plain FP64: the scale of the componentwise error metric."""
    return dgemm_naive(np.abs(np.asarray(A)), np.abs(np.asarray(B)), transa, transb)


def rel_err_vs_dd(C, A, B, transa="N", transb="N", alpha=1.0, beta=0.0, C0=None):
    """max_ij |C - C_dd| / (|alpha| |A||B| + |beta| |C0|)_ij, the componentwise error metric."""
    hi, lo = dgemm_dd(A, B, transa, transb, alpha, beta, C0)
    scale = abs(alpha) * abs_product(A, B, transa, transb)
    if C0 is not None and beta != 0.0:
        scale = scale + abs(beta) * np.abs(np.asarray(C0))
    diff = np.abs((np.asarray(C) - hi) - lo)
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.where(scale > 0, diff / np.where(scale > 0, scale, 1.0), np.where(diff > 0, np.inf, 0.0))
    return float(r.max()) if r.size else 0.0


# ----------------------------------------------------------------------------- selector
SEL_PARAMS = 6475


def mlp_loss_grad(theta, X, y):
    """O-mlp: mean cross-entropy and its FP64 gradient (BF16-rounded weights in the forward pass,
    straight-through gradient).  theta: float32[6475]; X: float32[B, 24]; y: int32[B]."""
    theta = np.ascontiguousarray(theta, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.int32)
    g = np.zeros(SEL_PARAMS)
    loss = _load().orc_mlp_loss_grad(_ptr(theta), _ptr(X), _ptr(y), int(len(y)), _ptr(g))
    return loss, g


def bf16_round(x: float) -> float:
    return float(_load().orc_bf16_round(float(x)))


def mlp_select(model: dict, feat, s_cap: int):
    """FP32 emulation of the GPU inference and decision.  model: mean, inv_std (float32[24]),
    W1, W2, W3 (uint16 BF16 bits), b1, b2, b3 (float32), thr, s_lo, fallback."""
    f = np.ascontiguousarray(feat, dtype=np.float32)
    arrs = [np.ascontiguousarray(model[k], dtype=dt) for k, dt in
            (("mean", np.float32), ("inv_std", np.float32), ("W1", np.uint16), ("b1", np.float32),
             ("W2", np.uint16), ("b2", np.float32), ("W3", np.uint16), ("b3", np.float32))]
    probs = np.zeros(11, dtype=np.float32)
    s = _load().orc_mlp_select(*[_ptr(a) for a in arrs], float(model["thr"]), int(model["s_lo"]),
                               int(model["fallback"]), _ptr(f), int(s_cap), _ptr(probs))
    return s, probs


def features(A, B, target, transa="N", transb="N"):
    """The selector's 24 features of op(A) op(B) from their definition (float32[24])."""
    A, B = _fortran(A, np.float64), _fortran(B, np.float64)
    m, k = _op_shape(transa, A)
    _, n = _op_shape(transb, B)
    out = np.zeros(24, dtype=np.float32)
    _load().orc_features(_b(transa), _b(transb), m, n, k, _ptr(A), max(A.shape[0], 1), _ptr(B), max(B.shape[0], 1),
                         float(target), _ptr(out))
    return out
