"""Host logic of the autotuner: launch orders and the cache signature."""
from paper_1203_1692_gb300 import autotune


def test_order_of():
    ns = [512, 8192, 1024, 8192, 600]
    assert autotune.order_of("given", ns) == [0, 1, 2, 3, 4]
    # largest first, ties in their given order
    assert autotune.order_of("largest_first", ns) == [1, 3, 2, 4, 0]


def test_signature_buckets_orders_and_taus():
    s1 = autotune.signature([512, 1000, 8000], [1e-7, 1e-7, 1e-8], "f16x3")
    # orders round to powers of two and sort; taus are a set
    s2 = autotune.signature([8192, 1024, 500], [1e-8, 1e-7], "f16x3")
    assert s1 == s2
    assert s1 != autotune.signature([512, 1000, 8000], [1e-7], "f16x3")
    assert s1 != autotune.signature([512, 1000, 8000], [1e-7, 1e-8], "tf32x3")


def test_choice_permutation_and_cache_lookup():
    c = autotune.Choice(leaf=32, order="largest_first", ms=1.0, slice=16)
    assert c.permutation([100, 300, 200]) == [1, 2, 0]
    key = autotune.signature([100], [1e-6], "bf16x3") + (
        tuple(autotune.LEAVES), tuple(autotune.ORDERS), tuple(autotune.SLICES))
    autotune._CACHE[key] = c
    try:
        assert autotune.cached([100], [1e-6], "bf16x3") is c
        assert autotune.cached([100], [1e-6], "f16x3") is None
    finally:
        del autotune._CACHE[key]


def _decay(A):
    from oracle import oracle as O
    return autotune.decay_from_pyramid(O.pyramid(A, 64), O.depth(A.shape[0], 64))


def test_decay_estimate_separates_decay_rates():
    """The norm-profile decay estimate (share of ||A||_F^2 on the 64 x 64
    diagonal leaves, read from a squared-norm pyramid): 1 for a
    block-diagonal matrix, about 64/n without decay, and ordered by the
    decay rate of exponential-decay matrices, so batches of equal orders but
    different decay get different signatures.  The pyramid here is the
    oracle's; on the GPU the library builds it."""
    import math
    import numpy as np
    import spamm_inputs as gen
    n = 512
    bd = np.zeros((n, n), dtype=np.float32)
    for k in range(0, n, 64):
        bd[k:k + 64, k:k + 64] = 1.0
    assert abs(_decay(bd) - 1.0) < 1e-12
    assert abs(_decay(gen.uniform_dense(n, seed=1)) - 64 / n) < 0.02
    e = [_decay(gen.exp_decay(n, lam, seed=2)) for lam in (0.5, 0.9, 0.99)]
    assert e[0] > e[1] > e[2]
    b = [int(round(math.log2(_decay(gen.exp_decay(n, lam, seed=2))))) for lam in (0.5, 0.99)]
    assert b[0] != b[1]
    s1 = autotune.signature([n, n], [1e-7], "f16x3", decay=b)
    s2 = autotune.signature([n, n], [1e-7], "f16x3", decay=[b[0], b[0]])
    assert s1 != s2
    assert autotune.signature([n], [1e-7], "f16x3", tier_bits=10) != \
        autotune.signature([n], [1e-7], "f16x3")
