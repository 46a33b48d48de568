"""Reading R11 on the CPU: the leaf squared norms are sums of exact squares
accumulated as FP32 pairs (each operand scaled by a power of two that
follows the largest exponent seen, squares split error-free, pairs added by
an error-free two-sum, folded into FP64 every eight rows).  This emulates
that arithmetic with IEEE float32 and float64 operations and checks it
against the correctly rounded sum of the exact squares: relative error far
below the 1e-12 the norm parity tests allow and the 1e-6 tie band."""
import math

import numpy as np
import pytest

F32 = np.float32


def _pow2f(k):
    return F32(2.0 ** k)


class _PairAcc:
    def __init__(self):
        self.hi = F32(0)
        self.lo = F32(0)
        self.sc = _pow2f(127)
        self.E = 0
        self.sum = 0.0

    def _add1(self, x):
        xs = F32(F32(x) * self.sc)
        p = F32(xs * xs)
        e = F32(float(xs) * float(xs) - float(p))   # exact: the two-product error
        t = F32(self.hi + p)
        bp = F32(t - self.hi)
        err = F32(F32(self.hi - F32(t - bp)) + F32(p - bp))
        self.hi = t
        self.lo = F32(self.lo + F32(err + e))

    def add4(self, v):
        m = max(int(np.asarray(x, dtype=F32).view(np.uint32) >> 23) & 0xFF for x in v)
        assert m != 0xFF
        if m > self.E:
            k = 2 * (self.E - m)
            f = _pow2f(k) if k >= -126 else F32(0)
            self.hi = F32(self.hi * f)
            self.lo = F32(self.lo * f)
            self.E = m
            self.sc = _pow2f(127 - self.E)
        for x in v:
            self._add1(x)

    def fold(self):
        self.sum = self.sum + (float(self.hi) + float(self.lo)) * 2.0 ** (2 * self.E - 254)
        self.hi = F32(0)
        self.lo = F32(0)


def _leaf_sum(block):
    """Squared norm of one b x b leaf as the kernel's threads form it: a
    thread per 4 columns down all rows (folding every 8 rows), then a tree
    of FP64 adds over the b/4 threads of the leaf."""
    b = block.shape[0]
    parts = []
    for c0 in range(0, b, 4):
        acc = _PairAcc()
        for r in range(b):
            acc.add4(block[r, c0:c0 + 4])
            if r % 8 == 7:
                acc.fold()
        if b % 8:
            acc.fold()
        parts.append(acc.sum)
    while len(parts) > 1:              # xor-shuffle reduction: pairs at distance 1, 2, ...
        half = len(parts) // 2
        parts = [parts[i] + parts[i + half] for i in range(half)]
    return parts[0]


def _exact(block):
    return math.fsum(float(x) * float(x) for x in block.astype(np.float64).ravel())


def _blocks():
    rng = np.random.default_rng(0)
    out = []
    out.append(rng.uniform(-1, 1, (16, 16)))
    out.append(rng.normal(size=(32, 32)) * 1e3)
    # magnitudes spread over 60 decades, the largest element last
    w = (rng.uniform(-1, 1, (16, 16)) * 10.0 ** rng.uniform(-30, 30, (16, 16)))
    w[-1, -1] = 3e33
    out.append(w)
    # subnormal and zero entries among normal ones
    s = rng.uniform(-1, 1, (16, 16)) * 1e-20
    s[::3, ::5] = 1e-44
    s[1::4] = 0.0
    out.append(s)
    out.append(rng.uniform(-1, 1, (64, 64)) * 10.0 ** rng.uniform(-5, 5, (64, 64)))
    return [x.astype(np.float32) for x in out]


@pytest.mark.parametrize("k", range(5))
def test_pair_accumulation_is_near_exact(k):
    block = _blocks()[k]
    got, want = _leaf_sum(block), _exact(block)
    assert want > 0
    assert abs(got - want) <= 1e-13 * want, (k, got, want)


def test_all_zero_leaf_is_zero():
    assert _leaf_sum(np.zeros((16, 16), dtype=np.float32)) == 0.0
