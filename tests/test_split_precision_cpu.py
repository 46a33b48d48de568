"""The arithmetic behind the split precisions' tolerances, on the CPU: each
operand split into a high and a low part of the MMA input format, the three
products hi*hi + hi*lo + lo*hi formed exactly (FP64) and compared with the
FP64 product.  This checks the representational error the tolerances in the
GPU parity tests are derived from (f16x3 and TF32x3: 1e-5; BF16x3: 1e-4),
not the GPU itself; the tensor core's FP32 accumulation adds at most a few
units of 2^-24 on top."""
import math

import numpy as np
import pytest

import spamm_inputs as gen


def _to_bf16(x):
    """Round float32 values to bfloat16 (round to nearest even), as float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _to_tf32(x):
    """Round float32 values to TF32 (10 fraction bits), ties away from zero."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x1000) & 0xFFFFE000
    return u.astype(np.uint32).view(np.float32)


def _split(x, fmt, scale=1.0):
    x = np.asarray(x, dtype=np.float32) * np.float32(scale)
    if fmt == "f16":
        hi = x.astype(np.float16).astype(np.float32)
        lo = (x - hi).astype(np.float16).astype(np.float32)
    elif fmt == "bf16":
        hi = _to_bf16(x)
        lo = _to_bf16(x - hi)
    else:
        hi = _to_tf32(x)
        lo = _to_tf32(x - hi)
    return hi.astype(np.float64), lo.astype(np.float64)


def _f16_scale(A, b):
    """2^k with k = 15 - e, the largest b x b leaf norm in [2^(e-1), 2^e)
    (from the exponent of the largest squared leaf norm, as the packs do)."""
    n = A.shape[0]
    nl = -(-n // b)
    P = np.zeros((nl * b, nl * b))
    P[:n, :n] = A.astype(np.float64) ** 2
    g2 = P.reshape(nl, b, nl, b).sum(axis=(1, 3)).max()
    if g2 <= 0:
        return 1.0
    E = math.frexp(g2)[1] - 1          # g2 in [2^E, 2^(E+1))
    k = 15 - ((E >> 1) + 1)
    return 2.0 ** max(-126, min(126, k))


def _split_product(A, B, fmt, b=32):
    sa = _f16_scale(A, b) if fmt == "f16" else 1.0
    sb = _f16_scale(B, b) if fmt == "f16" else 1.0
    ah, al = _split(A, fmt, sa)
    bh, bl = _split(B, fmt, sb)
    if fmt == "f16":
        # every scaled part fits fp16: no overflow to inf
        assert np.all(np.isfinite(ah)) and np.all(np.abs(ah) < 65504)
    return (ah @ bh + ah @ bl + al @ bh) / (sa * sb)


CASES = [("uniform", lambda: gen.uniform_dense(300, seed=1, symmetric=False)),
         ("exp", lambda: gen.exp_decay(300, 0.9, seed=2)),
         ("wide", lambda: (gen.uniform_dense(300, seed=3, symmetric=False).astype(np.float64)
                           * 10.0 ** np.random.default_rng(4).uniform(-12, 6, (300, 300))
                           ).astype(np.float32))]


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("fmt,bound", [("f16", 1e-6), ("tf32", 1e-6), ("bf16", 2e-5)])
def test_split_products_error(name, make, fmt, bound):
    A = make()
    B = gen.uniform_dense(300, seed=9, symmetric=False)
    exact = A.astype(np.float64) @ B.astype(np.float64)
    got = _split_product(A, B, fmt)
    err = np.abs(got - exact).max() / np.abs(exact).max()
    assert err <= bound, (name, fmt, err)


def test_f16_scale_keeps_tiny_and_huge_operands_in_range():
    rng = np.random.default_rng(5)
    for s in (2.0 ** 110, 2.0 ** -120, 2.0 ** -50):
        A = (rng.uniform(-1, 1, (64, 64)) * s).astype(np.float32)
        B = rng.uniform(-1, 1, (64, 64)).astype(np.float32)
        exact = A.astype(np.float64) @ B.astype(np.float64)
        got = _split_product(A, B, "f16", b=16)
        assert np.abs(got - exact).max() / np.abs(exact).max() <= 1e-6, s
