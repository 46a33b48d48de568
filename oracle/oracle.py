"""ctypes binding of the FP64 SpAMM oracle (oracle/spamm_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the package smoke check and
the benchmark's CPU-baseline leg, never by the library.  It does not import
the CUDA package and the CUDA package does not import it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "spamm_oracle.c")
LIB = os.path.join(HERE, "libspamm_oracle.so")

_c_i64 = ctypes.c_int64
_c_dbl = ctypes.c_double
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction, so the
    x86 and Arm builds round identically)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        L.oracle_depth.restype = ctypes.c_int
        L.oracle_depth.argtypes = [_c_i64, _c_i64]
        L.oracle_tier_offset.restype = _c_i64
        L.oracle_tier_offset.argtypes = [ctypes.c_int]
        L.oracle_pyramid_size.restype = _c_i64
        L.oracle_pyramid_size.argtypes = [ctypes.c_int]
        L.oracle_build_pyramid.restype = ctypes.c_int
        L.oracle_build_pyramid.argtypes = [_p, _c_i64, _c_i64, _c_i64, _p]
        L.oracle_keep.restype = ctypes.c_int
        L.oracle_keep.argtypes = [_c_dbl, _c_dbl, _c_dbl]
        L.oracle_cull_recursive.restype = _c_i64
        L.oracle_cull_recursive.argtypes = [_p, _p, ctypes.c_int, _c_dbl, _p, _c_i64, _p, _p]
        L.oracle_cull_linkless.restype = _c_i64
        L.oracle_cull_linkless.argtypes = [_p, _p, ctypes.c_int, _c_dbl, _p, _c_i64]
        L.oracle_morton.restype = ctypes.c_uint64
        L.oracle_morton.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        L.oracle_morton_decode.restype = None
        L.oracle_morton_decode.argtypes = [ctypes.c_uint64, _p, _p]
        for f in ("oracle_k_key_A", "oracle_k_key_B"):
            getattr(L, f).restype = ctypes.c_uint64
            getattr(L, f).argtypes = [ctypes.c_uint64]
        L.oracle_convolve.restype = ctypes.c_uint64
        L.oracle_convolve.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.oracle_multiply.restype = _c_i64
        L.oracle_multiply.argtypes = [_p, _c_i64, _p, _c_i64, _c_i64, _c_i64, _c_dbl, _c_dbl,
                                      _c_dbl, _p, _c_i64, _p, _c_i64, _p]
        L.oracle_multiply_sliced.restype = _c_i64
        L.oracle_multiply_sliced.argtypes = [_p, _c_i64, _p, _c_i64, _c_i64, _c_i64, _c_i64,
                                             _c_dbl, _c_dbl, ctypes.c_int, ctypes.c_int,
                                             _c_dbl, _c_dbl, _p, _c_i64, _p]
        L.oracle_round_sig.restype = _c_dbl
        L.oracle_round_sig.argtypes = [_c_dbl, ctypes.c_int, ctypes.c_int]
        L.oracle_multiply_tiered.restype = _c_i64
        L.oracle_multiply_tiered.argtypes = [_p, _c_i64, _p, _c_i64, _c_i64, _c_i64, _c_dbl,
                                             _c_dbl, ctypes.c_int, ctypes.c_int, _c_dbl, _c_dbl,
                                             _p, _c_i64, _p]
        L.oracle_sparsify.restype = _c_i64
        L.oracle_sparsify.argtypes = [_p, _c_i64, _c_i64, _c_i64, _c_dbl, _c_dbl, _p]
        L.oracle_block.restype = _c_i64
        L.oracle_block.argtypes = [_p, _c_i64, _p, _c_i64, _c_i64, _c_i64, _p, _p, _c_dbl,
                                   _c_dbl, ctypes.c_int, ctypes.c_int, _c_i64, _c_i64, _p]
        L.oracle_blocks.restype = _c_i64
        L.oracle_blocks.argtypes = [_p, _c_i64, _p, _c_i64, _c_i64, _c_i64, _p, _p, _c_dbl,
                                    _c_dbl, ctypes.c_int, ctypes.c_int, _p, _c_i64, _p]
        L.oracle_threads.restype = ctypes.c_int
        L.oracle_set_threads.restype = None
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _f32(A) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float32)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square matrix expected")
    return A


def depth(n: int, b: int) -> int:
    return lib().oracle_depth(n, b)


def tier_offset(t: int) -> int:
    return lib().oracle_tier_offset(t)


def pyramid(A, b: int) -> np.ndarray:
    """Squared-norm pyramid (all tiers, flat, tier t at (4^t-1)/3)."""
    A = _f32(A)
    n = A.shape[0]
    d = depth(n, b)
    out = np.empty(lib().oracle_pyramid_size(d), dtype=np.float64)
    lib().oracle_build_pyramid(_ptr(A), n, n, b, _ptr(out))
    return out


def tier(pyr: np.ndarray, t: int) -> np.ndarray:
    w = 1 << t
    o = tier_offset(t)
    return pyr[o:o + w * w].reshape(w, w)


def keep(nA2: float, nB2: float, tau: float) -> bool:
    return bool(lib().oracle_keep(nA2, nB2, tau))


def cull_recursive(pyrA, pyrB, d: int, tau: float):
    """(triples int32[m,3] as (I,K,J), cand[d+1], kept[d+1])."""
    cand = np.zeros(d + 1, dtype=np.int64)
    kept = np.zeros(d + 1, dtype=np.int64)
    cap = 1 << 16
    while True:
        out = np.empty((cap, 3), dtype=np.int32)
        m = lib().oracle_cull_recursive(_ptr(pyrA), _ptr(pyrB), d, tau, _ptr(out), cap,
                                        _ptr(cand), _ptr(kept))
        if m <= cap:
            return out[:m].copy(), cand, kept
        cap = int(m)


def cull_linkless(pyrA, pyrB, d: int, tau: float) -> np.ndarray:
    cap = 1 << 16
    while True:
        out = np.empty((cap, 3), dtype=np.int32)
        m = lib().oracle_cull_linkless(_ptr(pyrA), _ptr(pyrB), d, tau, _ptr(out), cap)
        if m < 0:
            raise MemoryError("oracle_cull_linkless")
        if m <= cap:
            return out[:m].copy()
        cap = int(m)


def morton(i: int, j: int) -> int:
    return int(lib().oracle_morton(i, j))


def morton_decode(l: int):
    i = ctypes.c_uint32()
    j = ctypes.c_uint32()
    lib().oracle_morton_decode(l, ctypes.addressof(i), ctypes.addressof(j))
    return i.value, j.value


def k_key_A(l: int) -> int:
    return int(lib().oracle_k_key_A(l))


def k_key_B(l: int) -> int:
    return int(lib().oracle_k_key_B(l))


def convolve(lA: int, lB: int) -> int:
    return int(lib().oracle_convolve(lA, lB))


class Result:
    """Output of :func:`multiply`."""

    def __init__(self, C, triples, cand, kept):
        self.C = C
        self.triples = triples
        self.cand = cand
        self.kept = kept


def multiply(A, B, b: int, tau: float, alpha: float = 1.0, beta: float = 0.0,
             C=None) -> Result:
    """C = alpha * SpAMM(A, B; b, tau) + beta * C, all in FP64."""
    A = _f32(A)
    B = _f32(B)
    n = A.shape[0]
    if B.shape != A.shape:
        raise ValueError("shape mismatch")
    d = depth(n, b)
    Cd = np.zeros((n, n), dtype=np.float64) if C is None else \
        np.ascontiguousarray(C, dtype=np.float64).copy()
    stats = np.zeros(2 * (d + 1), dtype=np.int64)
    cap = 1 << 16
    while True:
        out = np.empty((cap, 3), dtype=np.int32)
        m = lib().oracle_multiply(_ptr(A), n, _ptr(B), n, n, b, tau, alpha, beta,
                                  _ptr(Cd), n, _ptr(out), cap, _ptr(stats))
        if m == -2:          # capacity: grow to the exact count and redo
            pa, pb = pyramid(A, b), pyramid(B, b)
            cap = len(cull_recursive(pa, pb, d, tau)[0]) + 1
            continue
        if m < 0:
            raise RuntimeError(f"oracle_multiply failed ({m})")
        return Result(Cd, out[:m].copy(), stats[:d + 1].copy(), stats[d + 1:].copy())


def multiply_sliced(A, B, b: int, g: int, tau: float, alpha: float = 1.0, beta: float = 0.0,
                    C=None, tau_h: float = 0.0, p: int = 53, ties_away: bool = False):
    """C = alpha * SpAMM(A, B; b, tau) with the sub-leaf cull along k in
    slices of g (reading R14) + beta * C, in FP64; with tau_h > tau the
    precision of each kept leaf product chosen by its norm (R16).  Returns
    (C, kept leaf triples, kept slice products, tested slice products)."""
    A = _f32(A)
    B = _f32(B)
    n = A.shape[0]
    if B.shape != A.shape:
        raise ValueError("shape mismatch")
    Cd = np.zeros((n, n), dtype=np.float64) if C is None else \
        np.ascontiguousarray(C, dtype=np.float64).copy()
    stats = np.zeros(2, dtype=np.int64)
    m = lib().oracle_multiply_sliced(_ptr(A), n, _ptr(B), n, n, b, g, tau, tau_h, int(p),
                                     1 if ties_away else 0, alpha, beta, _ptr(Cd), n,
                                     _ptr(stats))
    if m < 0:
        raise RuntimeError(f"oracle_multiply_sliced failed ({m})")
    return Cd, int(m), int(stats[0]), int(stats[1])


# significant bits of the high part of each split precision, and whether
# its rounding breaks ties away from zero (TF32 conversion) or to even
HIGH_PART = {"f16x3": (11, False), "tf32x3": (11, True), "bf16x3": (8, False)}


def round_sig(x: float, p: int, ties_away: bool = False) -> float:
    """x rounded to p significant bits (unbounded exponent range)."""
    return float(lib().oracle_round_sig(float(x), int(p), 1 if ties_away else 0))


def multiply_tiered(A, B, b: int, tau: float, tau_h: float, p: int, ties_away: bool = False,
                    alpha: float = 1.0, beta: float = 0.0, C=None):
    """SpAMM at tau with the precision of each kept product chosen by its
    norm (reading R16): products with ||A_IK|| ||B_KJ|| >= tau_h exact,
    the others from operands rounded to p significant bits.  Returns (C in
    FP64, kept leaf triples, products formed exactly, products formed
    rounded)."""
    A = _f32(A)
    B = _f32(B)
    n = A.shape[0]
    if B.shape != A.shape:
        raise ValueError("shape mismatch")
    Cd = np.zeros((n, n), dtype=np.float64) if C is None else \
        np.ascontiguousarray(C, dtype=np.float64).copy()
    stats = np.zeros(2, dtype=np.int64)
    m = lib().oracle_multiply_tiered(_ptr(A), n, _ptr(B), n, n, b, tau, tau_h, int(p),
                                     1 if ties_away else 0, alpha, beta, _ptr(Cd), n,
                                     _ptr(stats))
    if m < 0:
        raise RuntimeError(f"oracle_multiply_tiered failed ({m})")
    return Cd, int(m), int(stats[0]), int(stats[1])


def sparsify(A, b: int, tau: float, norm2_max: float):
    """(A with the dropped leaves zeroed (float32), stored leaf count):
    a leaf is dropped iff ||A_IK||^2 * norm2_max < tau^2 or it is zero."""
    A = _f32(A)
    n = A.shape[0]
    out = np.empty((n, n), dtype=np.float32)
    m = lib().oracle_sparsify(_ptr(A), n, n, b, tau, norm2_max, _ptr(out))
    if m < 0:
        raise RuntimeError(f"oracle_sparsify failed ({m})")
    return out, int(m)


def blocks(A, B, b: int, tau: float, ij, pyrA=None, pyrB=None, tau_h: float = 0.0,
           p: int = 53, ties_away: bool = False):
    """Selected C blocks (no epilogue): array [len(ij), b, b] of FP64 and the
    total number of kept products over them; with tau_h > tau the precision
    of each kept product chosen by its norm (R16)."""
    A = _f32(A)
    B = _f32(B)
    n = A.shape[0]
    pa = pyramid(A, b) if pyrA is None else pyrA
    pb = pyramid(B, b) if pyrB is None else pyrB
    ij = np.ascontiguousarray(np.asarray(ij, dtype=np.int64).reshape(-1, 2))
    acc = np.zeros((len(ij), b, b), dtype=np.float64)
    tot = lib().oracle_blocks(_ptr(A), n, _ptr(B), n, n, b, _ptr(pa), _ptr(pb), tau, tau_h,
                              int(p), 1 if ties_away else 0, _ptr(ij), len(ij), _ptr(acc))
    return acc, int(tot)


def threads() -> int:
    return int(lib().oracle_threads())


def set_threads(t: int) -> None:
    lib().oracle_set_threads(t)
