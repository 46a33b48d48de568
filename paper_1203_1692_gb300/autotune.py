"""Autotuner for the leaf size and the schedule of batched SpAMM products.

The leaf size b sets how finely the cull of Sec. III works: small leaves
drop more of the product, large leaves give the tensor-core kernel longer
runs of work per step.  Which wins depends on n, on how fast the matrices
decay and on tau, so it is measured rather than modelled.  Every candidate
(leaf size, product order) runs the caller's own batch through
spamm_multiply_batched, event-timed on the context's stream after a
warm-up, and the fastest is kept.

The schedule candidates are the order of the products in the launch and,
when the caller allows it, the sub-leaf cull along k (16-wide slices).  The
persistent leaf kernel deals the concatenated list of C tiles out to its
blocks in turn, so the products at the end of the list make up the tail of
the launch; "largest_first" puts the big products first and leaves the small
ones to fill the tail.

Choices are cached in-process per signature: precision, precision tier,
tau, the products' orders rounded to powers of two, and a decay estimate
of each product from its norm profile (the share of the operand's squared
Frobenius norm held by its 64 x 64 diagonal blocks, as a power of two), so
a serving loop pays for a tuning run once per kind of batch and batches of
equal sizes but different decay are tuned apart.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

LEAVES = (16, 32, 64, 128)
ORDERS = ("given", "largest_first")
SLICES = (0, 16)          # sub-leaf cull along k: off, 16-wide slices (b >= 32)

_CACHE: dict = {}


@dataclass
class Choice:
    leaf: int
    order: str
    ms: float
    trials: dict = field(default_factory=dict)   # (leaf, order, slice) -> ms
    slice: int = 0

    def permutation(self, ns):
        return order_of(self.order, ns)


def order_of(order: str, ns):
    """Indices of the products in launch order."""
    idx = list(range(len(ns)))
    if order == "largest_first":
        idx.sort(key=lambda p: (-ns[p], p))
    return idx


def decay_from_pyramid(pyr, d: int) -> float:
    """Share of ||A||_F^2 held by the diagonal leaves, read from a squared-norm
    pyramid of depth d (tier t row-major at offset (4^t - 1) / 3, the root
    first): 1 for a block-diagonal matrix, about b / n without decay."""
    import numpy as np
    nb = 1 << d
    off = ((1 << (2 * d)) - 1) // 3
    leaf = np.asarray(pyr[off:off + nb * nb], dtype=np.float64).reshape(nb, nb)
    tot = float(pyr[0])
    return float(np.trace(leaf)) / tot if tot > 0 else 1.0


def decay_estimate(A, blk: int = 64) -> float:
    """The decay estimate of the square CUDA matrix A from its norm profile:
    the library's leaf-norm pyramid at leaf blk (an FP32 context, no packs),
    then the diagonal leaves' share of the root."""
    from . import Context
    ctx = Context(leaf=blk, precision="fp32")
    try:
        tree = ctx.build_norms(A)
        share = decay_from_pyramid(tree.norms(), tree.depth)
        tree.close()
    finally:
        ctx.close()
    return share


def decay_bucket(A) -> int:
    return int(round(math.log2(max(decay_estimate(A), 1e-30))))


def signature(ns, taus, precision: str, decay=None, tier_bits: int = 0):
    sig = (precision, int(tier_bits), tuple(sorted(round(math.log2(max(n, 1))) for n in ns)),
           tuple(sorted(set(float(t) for t in taus))))
    if decay is not None:
        sig += (tuple(sorted(decay)),)
    return sig


def cached(ns, taus, precision: str, leaves=LEAVES, orders=ORDERS, slices=SLICES, decay=None,
           tier_bits: int = 0):
    return _CACHE.get(signature(ns, taus, precision, decay, tier_bits) +
                      (tuple(leaves), tuple(orders), tuple(slices)))


def tune_batch(pairs, taus, precision: str = "tf32x3", leaves=LEAVES, orders=ORDERS,
               slices=SLICES, reps: int = 3, use_cache: bool = True,
               tier_bits: int = 0) -> Choice:
    """Pick (leaf, order, sub-leaf cull) for the batch of products ``pairs``
    = [(A, B), ...] (square float32 CUDA tensors) at thresholds ``taus``,
    under the precision tier ``tier_bits`` (0 = off).  The sub-leaf cull
    changes the approximation (it drops more), so it is a candidate only
    where the caller accepts that (``slices``)."""
    import torch
    from . import Context
    ns = [A.shape[0] for A, _ in pairs]
    decay = [decay_bucket(A) for A, _ in pairs]
    sig = signature(ns, taus, precision, decay, tier_bits) + (tuple(leaves), tuple(orders),
                                                              tuple(slices))
    if use_cache and sig in _CACHE:
        return _CACHE[sig]
    stream = torch.cuda.current_stream()
    trials = {}
    combos = [(b, sl) for b in leaves for sl in slices
              if sl == 0 or (precision != "fp32" and b >= 32)]
    for b, sl in combos:
        ctx = Context(leaf=b, precision=precision, checked=True, slice=sl, tier_bits=tier_bits)
        trees_a, trees_b = [], []
        for A, B in pairs:
            ta = ctx.build_norms(A)
            trees_a.append(ta)
            trees_b.append(ta if B is A else ctx.build_norms(B))
        Cs = [torch.empty_like(A) for A, _ in pairs]
        for order in orders:
            perm = order_of(order, ns)
            args = ([trees_a[p] for p in perm], [trees_b[p] for p in perm],
                    [taus[p] for p in perm], None, None, [Cs[p] for p in perm])
            ctx.set_checked(True)
            ctx.multiply_batched(*args)          # sizes the pools
            ctx.set_checked(False)
            ctx.multiply_batched(*args)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                ctx.multiply_batched(*args)
            e1.record(stream)
            torch.cuda.synchronize()
            ctx.stats()                          # raises if a timed call failed
            trials[(b, order, sl)] = e0.elapsed_time(e1) / reps
        for t in trees_a + trees_b:
            t.close()
        del Cs
        ctx.close()
        torch.cuda.empty_cache()
    (b, order, sl), ms = min(trials.items(), key=lambda kv: kv[1])
    choice = Choice(leaf=b, order=order, ms=ms, trials=trials, slice=sl)
    _CACHE[sig] = choice
    return choice
