"""GB300-native SpAMM engine (Sparse Approximate Matrix Multiply, Bock &
Challacombe).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/spamm.h``); this package only marshals PyTorch CUDA tensors into
that ABI.  There is no CPU fallback: without the built library every call
raises.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import (PRECISIONS, SpammError, spamm_build_norms, spamm_config_default,  # noqa: F401
                   spamm_create, spamm_destroy, spamm_multiply, spamm_multiply_batched,
                   spamm_multiply_host,
                   spamm_reserve, spamm_set_checked, spamm_set_stream, spamm_stats,
                   spamm_stats_item,
                   spamm_tree_destroy, spamm_tree_norms, spamm_tree_rebuild,
                   spamm_tree_rebuild_batched, spamm_tree_shape,
                   spamm_triples)

__all__ = ["Context", "Tree", "SpammError", "PRECISIONS", "load"]


def load():
    """Load the engine library (raises if it has not been built)."""
    return _abi.lib()


def _torch():
    import torch
    return torch


def _check_matrix(A):
    torch = _torch()
    if not isinstance(A, torch.Tensor) or not A.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if A.dtype != torch.float32 or A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("expected a square float32 matrix")
    if A.stride(1) != 1 or A.stride(0) < A.shape[0]:
        raise ValueError("expected row-major storage with leading dimension >= n")
    return A.shape[0], A.stride(0)


def _stats_dict(s) -> dict:
    """spamm_stats_t as a dict."""
    d = s.depth
    return {
        "status": s.status, "depth": d, "n": s.n, "leaf": s.leaf,
        "precision": s.precision, "tau": s.tau,
        "tier_candidates": list(s.tier_candidates[:d + 1]),
        "tier_kept": list(s.tier_kept[:d + 1]),
        "leaf_triples": s.leaf_triples, "tie_band": s.tie_band,
        "active_steps": s.active_steps, "tiles": s.tiles,
        "kept_flops": s.kept_flops, "dense_flops": s.dense_flops,
        "pool_bytes": s.pool_bytes, "pool_needed_bytes": s.pool_needed_bytes,
        "ms_symbolic": s.ms_symbolic, "ms_numeric": s.ms_numeric, "ms_total": s.ms_total,
        "ms_pack": s.ms_pack, "slice": s.slice, "slice_kept": s.slice_kept,
        "slice_tested": s.slice_tested,
        "packed_leaves_a": s.packed_leaves_a, "packed_leaves_b": s.packed_leaves_b,
        "hi_products": s.hi_products, "tie_band_hi": s.tie_band_hi,
        "kept_flops_clipped": s.kept_flops_clipped,
    }


class Tree:
    """Norm quadtree of a matrix (holds a reference to the matrix, unless it
    is a sparsified tree, which holds its own copy of the kept leaves)."""

    def __init__(self, ctx: "Context", A, sparsify=None):
        n, lda = _check_matrix(A)
        self.ctx = ctx
        self.n = n
        self.device = A.device
        if sparsify is None:
            self.A = A
            self.handle = spamm_build_norms(ctx.handle, A.data_ptr(), n, lda)
        else:
            tau, partner_norm2 = sparsify
            self.A = None
            self.handle = _abi.spamm_sparsify(ctx.handle, A.data_ptr(), n, lda, tau,
                                              partner_norm2)
        self.depth, self.nodes = spamm_tree_shape(self.handle)

    @property
    def bytes(self) -> int:
        return _abi.spamm_tree_bytes(self.handle)[0]

    @property
    def stored_leaves(self) -> int:
        """Kept leaves of a sparsified tree (-1 for a dense tree)."""
        return _abi.spamm_tree_bytes(self.handle)[1]

    def rebuild(self, A):
        n, lda = _check_matrix(A)
        if n != self.n:
            raise ValueError("rebuild needs the same n")
        self.A = A
        spamm_tree_rebuild(self.ctx.handle, self.handle, A.data_ptr(), lda)

    def resparsify(self, A, tau: float, partner_norm2: float = 0.0):
        """Sparsify new contents A (same n) into this sparsified tree, reusing
        its device storage while the new bands fit."""
        n, lda = _check_matrix(A)
        if n != self.n:
            raise ValueError("resparsify needs the same n")
        _abi.spamm_sparsify_into(self.ctx.handle, self.handle, A.data_ptr(), lda, tau,
                                 partner_norm2)

    def norms(self) -> np.ndarray:
        out = np.empty(self.nodes, dtype=np.float64)
        spamm_tree_norms(self.ctx.handle, self.handle, out.ctypes.data, self.nodes)
        return out

    def close(self):
        if self.handle:
            spamm_tree_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """A SpAMM context on the current CUDA device and stream."""

    def __init__(self, leaf: int = 16, precision: str = "fp32", tie_rel: float = 1e-6,
                 pool_bytes: int = 0, checked: bool = True, stream=None, slice: int = 0,
                 tier_bits: int = 0, staged: bool = False):
        torch = _torch()
        cfg = spamm_config_default()
        cfg.leaf = leaf
        cfg.slice = slice
        cfg.tier_bits = tier_bits
        cfg.staged = 1 if staged else 0
        cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        cfg.tie_rel = tie_rel
        cfg.pool_bytes = pool_bytes
        cfg.checked = 1 if checked else 0
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = spamm_create(self.stream.cuda_stream, cfg)
        self.leaf = leaf
        self.slice = slice
        self.tier_bits = tier_bits
        self.precision = precision

    def build_norms(self, A) -> Tree:
        return Tree(self, A)

    def sparsify(self, A, tau: float, partner_norm2: float = 0.0) -> Tree:
        """A sparsified tree of A: leaves whose product with max(||A||_F^2,
        partner_norm2) fails the SpAMM test at tau are dropped, the rest
        stored band by band (the paper's drop tolerance epsilon = tau /
        max(||A||_F, ||B||_F) when partner_norm2 = ||B||_F^2)."""
        return Tree(self, A, sparsify=(tau, partner_norm2))

    def tree_footprint(self, n: int) -> int:
        """Device bytes of a tree of order n under this configuration."""
        return _abi.spamm_tree_footprint(self.handle, n)

    def multiply(self, A: Tree, B: Tree, tau: float, alpha: float = 1.0, beta: float = 0.0,
                 C=None):
        torch = _torch()
        if C is None:
            C = torch.empty((A.n, A.n), dtype=torch.float32, device=A.device)
        n, ldc = _check_matrix(C)
        if n != A.n:
            raise ValueError("C has the wrong size")
        spamm_multiply(self.handle, A.handle, B.handle, tau, alpha, beta, C.data_ptr(), ldc)
        return C

    def rebuild_batched(self, trees, mats):
        """Tree.rebuild for many trees at once (the norm builds overlap on
        the context's side streams)."""
        ldas = []
        for t, A in zip(trees, mats):
            n, lda = _check_matrix(A)
            if n != t.n:
                raise ValueError("rebuild needs the same n")
            ldas.append(lda)
        spamm_tree_rebuild_batched(self.handle, [t.handle for t in trees],
                                   [A.data_ptr() for A in mats], ldas)
        for t, A in zip(trees, mats):
            t.A = A

    def multiply_batched(self, As, Bs, taus, alphas=None, betas=None, Cs=None):
        """Independent products C[p] = alpha[p] SpAMM(A[p], B[p]; tau[p]) +
        beta[p] C[p] in one call (one persistent leaf launch on the
        tensor-core precisions).  ``As``/``Bs`` are Trees; scalars broadcast."""
        torch = _torch()
        count = len(As)
        def bcast(x, default):
            if x is None:
                x = default
            return list(x) if isinstance(x, (list, tuple)) else [x] * count
        taus = bcast(taus, 0.0)
        alphas = bcast(alphas, 1.0)
        betas = bcast(betas, 0.0)
        if Cs is None:
            Cs = [torch.empty((a.n, a.n), dtype=torch.float32, device=a.device) for a in As]
        ldcs = []
        for a, C in zip(As, Cs):
            n, ldc = _check_matrix(C)
            if n != a.n:
                raise ValueError("C has the wrong size")
            ldcs.append(ldc)
        spamm_multiply_batched(self.handle, [a.handle for a in As], [b.handle for b in Bs],
                               taus, alphas, betas, [C.data_ptr() for C in Cs], ldcs)
        return Cs

    def multiply_host(self, A: np.ndarray, B, tau: float, alpha: float = 1.0,
                      beta: float = 0.0, C=None) -> np.ndarray:
        """End to end from host arrays (numpy float32, C-contiguous, or pinned
        torch CPU tensors)."""
        def ptr(x):
            if hasattr(x, "data_ptr"):
                return x.data_ptr()
            return x.ctypes.data
        n = A.shape[0]
        if C is None:
            C = np.zeros((n, n), dtype=np.float32)
        spamm_multiply_host(self.handle, ptr(A), ptr(B) if B is not None else None, n, tau,
                            alpha, beta, ptr(C))
        return C

    def set_checked(self, checked: bool):
        spamm_set_checked(self.handle, checked)

    def reserve(self, pool_bytes: int):
        spamm_reserve(self.handle, pool_bytes)

    def set_wait_limit(self, wait_ns: int):
        """Bound of the leaf kernel's pipeline waits (ns; 0 = the default 1 s)."""
        _abi.check(_abi.lib().spamm_set_wait_limit(self.handle, int(wait_ns)), self.handle)

    def stats(self, raise_on_error: bool = True) -> dict:
        return _stats_dict(spamm_stats(self.handle, raise_on_error))

    def stats_item(self, index: int, raise_on_error: bool = True) -> dict:
        """Statistics of product ``index`` of the last batched multiply."""
        return _stats_dict(spamm_stats_item(self.handle, index, raise_on_error))

    def per_product_flops(self, count: int) -> list:
        """Kept flops of each product of the last batched multiply (over the
        leaves' extents inside the matrices)."""
        return [spamm_stats_item(self.handle, p).kept_flops_clipped for p in range(count)]

    def cull_flat(self, A: Tree, B: Tree, tau: float, triples: bool = True):
        """The flat, norm-sorted enumeration (Algorithm 1) on the GPU:
        (rows (I, K, J) sorted by (I, J, K) or None, count, device ms)."""
        if not triples:
            cnt, ms = _abi.spamm_cull_flat(self.handle, A.handle, B.handle, tau, 0, 0)
            return None, cnt, ms
        cnt, _ = _abi.spamm_cull_flat(self.handle, A.handle, B.handle, tau, 0, 0)
        out = np.empty((max(cnt, 1), 3), dtype=np.int32)
        cnt, ms = _abi.spamm_cull_flat(self.handle, A.handle, B.handle, tau, out.ctypes.data,
                                       cnt)
        return out[:cnt], cnt, ms

    def triples(self, hi: bool = False) -> np.ndarray:
        """Surviving leaf triples (I, K, J) of the last multiply; with hi,
        only those that ran with the full split precision (tier_bits)."""
        f = _abi.spamm_triples_hi if hi else spamm_triples
        count = ctypes.c_int64()
        getattr(_abi.lib(), "spamm_triples_hi" if hi else "spamm_triples")(
            self.handle, None, 0, ctypes.byref(count))
        out = np.empty((max(count.value, 1), 3), dtype=np.int32)
        m = f(self.handle, out.ctypes.data, count.value)
        return out[:m]

    def close(self):
        if self.handle:
            spamm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
