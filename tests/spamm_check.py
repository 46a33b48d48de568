"""Helpers that compare the CUDA path (through the C ABI) with the FP64
oracle.  Used by the GPU tests, the package smoke check and the benchmark's
parity gate."""
from __future__ import annotations

import math

import numpy as np

from oracle import oracle as O


def as_set(tr) -> set:
    return set(map(tuple, np.asarray(tr).reshape(-1, 3).tolist()))


def tie_band(pyrA, pyrB, d, tau, rel=1e-6, triples=None):
    """Leaf triples whose norm product lies within rel * tau of tau (the
    oracle's norms).  ``triples`` restricts the check to given triples."""
    la = O.tier(pyrA, d)
    lb = O.tier(pyrB, d)
    out = set()
    if triples is None:
        w = la.shape[0]
        for I in range(w):
            for K in range(w):
                if la[I, K] <= 0:
                    continue
                for J in range(w):
                    p = la[I, K] * lb[K, J]
                    if p > 0 and abs(math.sqrt(p) - tau) <= rel * tau:
                        out.add((I, K, J))
        return out
    for (I, K, J) in triples:
        p = la[I, K] * lb[K, J]
        if p > 0 and abs(math.sqrt(p) - tau) <= rel * tau:
            out.add((I, K, J))
    return out


def compare_triples(gpu, orc, pyrA, pyrB, d, tau, rel=1e-6):
    """Bit-exact set equality outside the tie band; returns the number of
    disagreeing triples (all inside the band) for reporting."""
    g, o = as_set(gpu), as_set(orc)
    diff = g ^ o
    band = tie_band(pyrA, pyrB, d, tau, rel, triples=diff)
    assert diff <= band, f"{len(diff - band)} triples differ outside the tie band"
    return len(diff)


def rel_max_err(C, ref) -> float:
    ref = np.asarray(ref, dtype=np.float64)
    den = np.abs(ref).max()
    num = np.abs(np.asarray(C, dtype=np.float64) - ref).max()
    return float(num / den) if den > 0 else float(num)


def sample_blocks(n, b, count, seed=0, diag=True):
    nl = -(-n // b)
    rng = np.random.default_rng(seed)
    ij = [(int(i), int(j)) for i, j in rng.integers(0, nl, size=(count, 2))]
    if diag:
        ij += [(0, 0), (nl - 1, nl - 1), (nl // 2, nl // 2), (nl // 2, max(0, nl // 2 - 1))]
    return sorted(set(ij))


def blocks_from(C, ij, b, n):
    out = np.zeros((len(ij), b, b), dtype=np.float64)
    for q, (I, J) in enumerate(ij):
        blk = np.asarray(C[I * b:min(n, (I + 1) * b), J * b:min(n, (J + 1) * b)], dtype=np.float64)
        out[q, :blk.shape[0], :blk.shape[1]] = blk
    return out


def _keys(tr) -> np.ndarray:
    t = np.asarray(tr, dtype=np.int64).reshape(-1, 3)
    return np.unique((t[:, 0] << 42) | (t[:, 1] << 21) | t[:, 2])


def compare_triples_large(gpu, orc, pyrA, pyrB, d, tau, rel=1e-6):
    """compare_triples for millions of triples: the two sets as sorted
    integer keys, their symmetric difference checked against the tie band
    with the oracle's leaf norms.  Returns the number of disagreeing
    triples (all inside the band)."""
    g, o = _keys(gpu), _keys(orc)
    assert len(g) == len(np.asarray(gpu).reshape(-1, 3)), "duplicate GPU triples"
    diff = np.setxor1d(g, o, assume_unique=True)
    if diff.size == 0:
        return 0
    la = O.tier(pyrA, d)
    lb = O.tier(pyrB, d)
    I, K, J = diff >> 42, (diff >> 21) & ((1 << 21) - 1), diff & ((1 << 21) - 1)
    p = la[I, K] * lb[K, J]
    inside = (p > 0) & (np.abs(np.sqrt(p) - tau) <= rel * tau)
    assert inside.all(), f"{int((~inside).sum())} triples differ outside the tie band"
    return int(diff.size)
