"""The exponential-decay generator of ``generators.exp_decay`` evaluated with
PyTorch tensor ops on any device, so large batches of inputs (hundreds of
millions of elements) are made where they are used instead of on the host.

It draws the same counter-based SplitMix64 numbers as the numpy version and
gives the same float32 matrix bit for bit:

- 64-bit unsigned arithmetic is done in int64, whose add and multiply wrap
  modulo 2^64 exactly like uint64; right shifts are made logical by masking
  off the sign-extended bits;
- lambda^|i-j| is not recomputed on the device: the host evaluates
  ``exp(log(lambda) * d)`` with numpy for every distance d < n (the same
  expression, so the same float64 values) and the device gathers it;
- the uniform draw, the product and the float32 rounding are single IEEE
  operations, identical on every device.

No SpAMM arithmetic lives here.
"""
from __future__ import annotations

import math

import numpy as np

from .generators import _MAX_INDEX, _seed_base

_SLAB = 1 << 24          # elements generated per slab on the device


def _as_i64(u: int) -> int:
    """The int64 with the bit pattern of the uint64 ``u``."""
    u &= (1 << 64) - 1
    return u - (1 << 64) if u >= (1 << 63) else u


_GAMMA = _as_i64(0x9E3779B97F4A7C15)
_M1 = _as_i64(0xBF58476D1CE4E5B9)
_M2 = _as_i64(0x94D049BB133111EB)


def _srl(z, k: int):
    """Logical right shift of int64 bit patterns."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def _mix64(z):
    z = z ^ _srl(z, 30)
    z = z * _M1
    z = z ^ _srl(z, 27)
    z = z * _M2
    return z ^ _srl(z, 31)


def exp_decay(n: int, lam: float = 0.9, seed: int = 0, device="cuda", out=None):
    """a_ij = u_ij * lam^|i-j| as ``generators.exp_decay(n, lam, seed)``,
    returned as an n x n float32 tensor on ``device`` (or written to
    ``out``)."""
    import torch
    if n <= 0 or n > _MAX_INDEX:
        raise ValueError(f"matrix order {n} out of range")
    dev = torch.device(device)
    if out is None:
        out = torch.empty((n, n), dtype=torch.float32, device=dev)
    loglam = math.log(lam)
    powers = torch.from_numpy(np.exp(loglam * np.arange(n, dtype=np.float64))).to(dev)
    base = _as_i64(int(_seed_base(seed)))
    j = torch.arange(n, dtype=torch.int64, device=dev)[None, :]
    rows = max(1, _SLAB // n)
    for r0 in range(0, n, rows):
        r1 = min(n, r0 + rows)
        i = torch.arange(r0, r1, dtype=torch.int64, device=dev)[:, None]
        lo = torch.minimum(i, j)
        hi = torch.maximum(i, j)
        c = (lo << 28) | hi                                  # stream 0
        z = _mix64(base + (c + 1) * _GAMMA)
        u = (_srl(z, 11).to(torch.float64) + 0.5) * (2.0 ** -52) - 1.0
        out[r0:r1] = (u * powers[(i - j).abs()]).to(torch.float32)
    return out


def algebraic_decay(n: int, seed: int = 0, device="cuda", out=None):
    """a_ij = s_ij / (|i-j|^2 + 1), s_ij = +-1, as
    ``generators.algebraic_decay(n, seed)``: the same SplitMix64 draws
    (stream 3), the sign from their top bit, the quotient in float64 and one
    rounding to float32, so the same matrix bit for bit."""
    import torch
    if n <= 0 or n > _MAX_INDEX:
        raise ValueError(f"matrix order {n} out of range")
    dev = torch.device(device)
    if out is None:
        out = torch.empty((n, n), dtype=torch.float32, device=dev)
    base = _as_i64(int(_seed_base(seed)))
    j = torch.arange(n, dtype=torch.int64, device=dev)[None, :]
    rows = max(1, _SLAB // n)
    for r0 in range(0, n, rows):
        r1 = min(n, r0 + rows)
        i = torch.arange(r0, r1, dtype=torch.int64, device=dev)[:, None]
        lo = torch.minimum(i, j)
        hi = torch.maximum(i, j)
        c = (3 << 56) | (lo << 28) | hi                      # stream 3
        z = _mix64(base + (c + 1) * _GAMMA)
        s = torch.where(z < 0, -1.0, 1.0).to(torch.float64)  # top bit set: -1
        d = (i - j).abs().to(torch.float64)
        out[r0:r1] = (s / (d * d + 1.0)).to(torch.float32)
    return out
