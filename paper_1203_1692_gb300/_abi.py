"""ctypes binding of the C ABI in include/spamm.h.

Argument marshalling only: every step of the SpAMM path runs in the CUDA
kernels of ``libspamm_gb300.so``.  If the library has not been built the
import fails loudly; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspamm_gb300.so")

SPAMM_OK = 0
SPAMM_ERR_INVALID_ARG = 1
SPAMM_ERR_NONFINITE = 2
SPAMM_ERR_CAPACITY = 3
SPAMM_ERR_OOM = 4
SPAMM_ERR_TIMEOUT = 5
SPAMM_ERR_UNSUPPORTED = 6
SPAMM_ERR_CUDA = 7
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "NONFINITE", 3: "CAPACITY", 4: "OOM",
                5: "TIMEOUT", 6: "UNSUPPORTED", 7: "CUDA"}

SPAMM_PREC_FP32 = 0
SPAMM_PREC_TF32X3 = 1
SPAMM_PREC_TF32 = 2
SPAMM_PREC_BF16X3 = 3
SPAMM_PREC_F16X3 = 4
PRECISIONS = {"fp32": 0, "tf32x3": 1, "tf32": 2, "bf16x3": 3, "f16x3": 4}

SPAMM_MAX_TIERS = 32


class spamm_config(ctypes.Structure):
    _fields_ = [("leaf", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("tie_rel", ctypes.c_double), ("pool_bytes", ctypes.c_int64),
                ("checked", ctypes.c_int32), ("slice", ctypes.c_int32),
                ("tier_bits", ctypes.c_int32), ("staged", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


class spamm_stats_t(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("depth", ctypes.c_int32), ("n", ctypes.c_int64),
                ("leaf", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("tau", ctypes.c_double),
                ("tier_candidates", ctypes.c_int64 * SPAMM_MAX_TIERS),
                ("tier_kept", ctypes.c_int64 * SPAMM_MAX_TIERS),
                ("leaf_triples", ctypes.c_int64), ("tie_band", ctypes.c_int64),
                ("active_steps", ctypes.c_int64), ("tiles", ctypes.c_int64),
                ("kept_flops", ctypes.c_double), ("dense_flops", ctypes.c_double),
                ("pool_bytes", ctypes.c_int64), ("pool_needed_bytes", ctypes.c_int64),
                ("ms_symbolic", ctypes.c_float), ("ms_numeric", ctypes.c_float),
                ("ms_total", ctypes.c_float), ("ms_pack", ctypes.c_float),
                ("slice", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("slice_kept", ctypes.c_int64), ("slice_tested", ctypes.c_int64),
                ("packed_leaves_a", ctypes.c_int64), ("packed_leaves_b", ctypes.c_int64),
                ("hi_products", ctypes.c_int64), ("tie_band_hi", ctypes.c_int64),
                ("kept_flops_clipped", ctypes.c_double)]


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_flt = ctypes.c_float

# name -> (restype, argtypes); every symbol include/spamm.h declares
SIGNATURES = {
    "spamm_config_default": (None, [ctypes.POINTER(spamm_config)]),
    "spamm_create": (_i32, [ctypes.POINTER(_vp), _vp, ctypes.POINTER(spamm_config)]),
    "spamm_destroy": (_i32, [_vp]),
    "spamm_set_stream": (_i32, [_vp, _vp]),
    "spamm_set_checked": (_i32, [_vp, _i32]),
    "spamm_reserve": (_i32, [_vp, _i64]),
    "spamm_set_wait_limit": (_i32, [_vp, _i64]),
    "spamm_last_error": (ctypes.c_char_p, [_vp]),
    "spamm_build_norms": (_i32, [_vp, _vp, _i64, _i64, ctypes.POINTER(_vp)]),
    "spamm_tree_rebuild": (_i32, [_vp, _vp, _vp, _i64]),
    "spamm_tree_rebuild_batched": (_i32, [_vp, _i32, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                          ctypes.POINTER(_i64)]),
    "spamm_tree_destroy": (_i32, [_vp]),
    "spamm_tree_shape": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i64)]),
    "spamm_tree_footprint": (_i32, [_vp, _i64, ctypes.POINTER(_i64)]),
    "spamm_sparsify": (_i32, [_vp, _vp, _i64, _i64, _dbl, _dbl, ctypes.POINTER(_vp)]),
    "spamm_sparsify_into": (_i32, [_vp, _vp, _vp, _i64, _dbl, _dbl]),
    "spamm_tree_bytes": (_i32, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "spamm_tree_norms": (_i32, [_vp, _vp, _vp, _i64]),
    "spamm_multiply": (_i32, [_vp, _vp, _vp, _dbl, _flt, _flt, _vp, _i64]),
    "spamm_multiply_batched": (_i32, [_vp, _i32, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                      ctypes.POINTER(_dbl), ctypes.POINTER(_flt),
                                      ctypes.POINTER(_flt), ctypes.POINTER(_vp),
                                      ctypes.POINTER(_i64)]),
    "spamm_multiply_host": (_i32, [_vp, _vp, _vp, _i64, _dbl, _flt, _flt, _vp]),
    "spamm_stats": (_i32, [_vp, ctypes.POINTER(spamm_stats_t)]),
    "spamm_stats_item": (_i32, [_vp, _i32, ctypes.POINTER(spamm_stats_t)]),
    "spamm_triples": (_i32, [_vp, _vp, _i64, ctypes.POINTER(_i64)]),
    "spamm_triples_hi": (_i32, [_vp, _vp, _i64, ctypes.POINTER(_i64)]),
    "spamm_cull_flat": (_i32, [_vp, _vp, _vp, _dbl, _vp, _i64, ctypes.POINTER(_i64),
                               ctypes.POINTER(_flt)]),
    "spamm_multiply_static": (_i32, [_vp, _i64, _vp, _i64, _i64, _dbl, _flt, _flt, _vp, _i64,
                                     _vp, _vp]),
}

_lib = None


def lib():
    """The loaded engine library; raises if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1203_1692_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class SpammError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, ctx=None) -> None:
    if status != SPAMM_OK:
        msg = lib().spamm_last_error(ctx).decode() if ctx else ""
        raise SpammError(status, msg)


# Thin same-name wrappers -------------------------------------------------

def spamm_config_default() -> spamm_config:
    c = spamm_config()
    lib().spamm_config_default(ctypes.byref(c))
    return c


def spamm_create(stream: int, cfg: spamm_config):
    h = _vp()
    check(lib().spamm_create(ctypes.byref(h), _vp(stream), ctypes.byref(cfg)))
    return h


def spamm_destroy(ctx) -> None:
    check(lib().spamm_destroy(ctx))


def spamm_set_stream(ctx, stream: int) -> None:
    check(lib().spamm_set_stream(ctx, _vp(stream)), ctx)


def spamm_set_checked(ctx, checked: bool) -> None:
    check(lib().spamm_set_checked(ctx, 1 if checked else 0), ctx)


def spamm_reserve(ctx, pool_bytes: int) -> None:
    check(lib().spamm_reserve(ctx, int(pool_bytes)), ctx)


def spamm_build_norms(ctx, A_ptr: int, n: int, lda: int):
    h = _vp()
    check(lib().spamm_build_norms(ctx, _vp(A_ptr), n, lda, ctypes.byref(h)), ctx)
    return h


def spamm_tree_rebuild(ctx, tree, A_ptr: int, lda: int) -> None:
    check(lib().spamm_tree_rebuild(ctx, tree, _vp(A_ptr), lda), ctx)


def spamm_tree_rebuild_batched(ctx, trees, A_ptrs, ldas) -> None:
    count = len(trees)
    if not (len(A_ptrs) == len(ldas) == count):
        raise ValueError("batched arguments differ in length")
    t = (_vp * max(count, 1))(*trees)
    a = (_vp * max(count, 1))(*[_vp(x) for x in A_ptrs])
    ld = (_i64 * max(count, 1))(*[int(x) for x in ldas])
    check(lib().spamm_tree_rebuild_batched(ctx, count, t, a, ld), ctx)


def spamm_tree_destroy(tree) -> None:
    check(lib().spamm_tree_destroy(tree))


def spamm_tree_shape(tree):
    d = _i32()
    m = _i64()
    check(lib().spamm_tree_shape(tree, ctypes.byref(d), ctypes.byref(m)))
    return d.value, m.value


def spamm_tree_footprint(ctx, n: int) -> int:
    out = _i64()
    check(lib().spamm_tree_footprint(ctx, n, ctypes.byref(out)), ctx)
    return out.value


def spamm_sparsify(ctx, A_ptr: int, n: int, lda: int, tau: float, partner_norm2: float):
    h = _vp()
    check(lib().spamm_sparsify(ctx, _vp(A_ptr), n, lda, float(tau), float(partner_norm2),
                               ctypes.byref(h)), ctx)
    return h


def spamm_sparsify_into(ctx, tree, A_ptr: int, lda: int, tau: float, partner_norm2: float):
    check(lib().spamm_sparsify_into(ctx, tree, _vp(A_ptr), lda, float(tau),
                                    float(partner_norm2)), ctx)


def spamm_tree_bytes(tree):
    b = _i64()
    st = _i64()
    check(lib().spamm_tree_bytes(tree, ctypes.byref(b), ctypes.byref(st)))
    return b.value, st.value


def spamm_tree_norms(ctx, tree, out_ptr: int, count: int) -> None:
    check(lib().spamm_tree_norms(ctx, tree, _vp(out_ptr), count), ctx)


def spamm_multiply(ctx, A_tree, B_tree, tau: float, alpha: float, beta: float, C_ptr: int,
                   ldc: int) -> int:
    st = lib().spamm_multiply(ctx, A_tree, B_tree, float(tau), float(alpha), float(beta),
                              _vp(C_ptr), ldc)
    check(st, ctx)
    return st


def spamm_multiply_batched(ctx, A_trees, B_trees, taus, alphas, betas, C_ptrs, ldcs) -> None:
    """C[p] = alpha[p] SpAMM(A[p], B[p]; tau[p]) + beta[p] C[p] for every p."""
    count = len(A_trees)
    if not (len(B_trees) == len(taus) == len(alphas) == len(betas) == len(C_ptrs) == len(ldcs)
            == count):
        raise ValueError("batched arguments differ in length")
    a = (_vp * max(count, 1))(*A_trees)
    b = (_vp * max(count, 1))(*B_trees)
    t = (_dbl * max(count, 1))(*[float(x) for x in taus])
    al = (_flt * max(count, 1))(*[float(x) for x in alphas])
    be = (_flt * max(count, 1))(*[float(x) for x in betas])
    c = (_vp * max(count, 1))(*[_vp(x) for x in C_ptrs])
    ld = (_i64 * max(count, 1))(*[int(x) for x in ldcs])
    check(lib().spamm_multiply_batched(ctx, count, a, b, t, al, be, c, ld), ctx)


def spamm_multiply_host(ctx, A_ptr: int, B_ptr, n: int, tau: float, alpha: float,
                        beta: float, C_ptr: int) -> None:
    check(lib().spamm_multiply_host(ctx, _vp(A_ptr), _vp(B_ptr) if B_ptr else None, n,
                                    float(tau), float(alpha), float(beta), _vp(C_ptr)), ctx)


def spamm_stats(ctx, raise_on_error: bool = True) -> spamm_stats_t:
    s = spamm_stats_t()
    st = lib().spamm_stats(ctx, ctypes.byref(s))
    if raise_on_error:
        check(st, ctx)
    return s


def spamm_stats_item(ctx, index: int, raise_on_error: bool = True) -> spamm_stats_t:
    s = spamm_stats_t()
    st = lib().spamm_stats_item(ctx, index, ctypes.byref(s))
    if raise_on_error:
        check(st, ctx)
    return s


def spamm_triples(ctx, out_ptr: int, cap: int) -> int:
    cnt = _i64()
    check(lib().spamm_triples(ctx, _vp(out_ptr), cap, ctypes.byref(cnt)), ctx)
    return cnt.value


def spamm_triples_hi(ctx, out_ptr: int, cap: int) -> int:
    cnt = _i64()
    check(lib().spamm_triples_hi(ctx, _vp(out_ptr), cap, ctypes.byref(cnt)), ctx)
    return cnt.value


def spamm_cull_flat(ctx, A_tree, B_tree, tau: float, out_ptr: int, cap: int):
    """(count, ms) of the flat enumeration; rows (I, K, J) into out_ptr."""
    cnt = _i64()
    ms = _flt()
    check(lib().spamm_cull_flat(ctx, A_tree, B_tree, float(tau), _vp(out_ptr) if out_ptr else None,
                                cap, ctypes.byref(cnt), ctypes.byref(ms)), ctx)
    return cnt.value, ms.value


def spamm_multiply_static(A_ptr: int, lda: int, B_ptr: int, ldb: int, n: int, tau: float,
                          alpha: float, beta: float, C_ptr: int, ldc: int, stream: int,
                          status_ptr: int = 0) -> None:
    """The allocation-free FP32 product (all scratch in a static device
    array, n <= 4096); see include/spamm.h."""
    check(lib().spamm_multiply_static(_vp(A_ptr), lda, _vp(B_ptr), ldb, n, float(tau),
                                      float(alpha), float(beta), _vp(C_ptr), ldc,
                                      _vp(stream), _vp(status_ptr) if status_ptr else None))
