"""Seeded synthetic inputs for SpAMM workloads.

This module is shared by the FP64 oracle (test infrastructure) and the CUDA
path.  It holds only random-number generation and the decay profiles that
define the synthetic matrices; none of the SpAMM arithmetic (norms, culling,
products) lives here.

Random numbers come from a counter-based SplitMix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): the value for
a counter c under seed s is the SplitMix64 output function applied to
``base(s) + (c + 1) * GAMMA``.  A matrix element (i, j) uses the counter
``(stream << 56) | (min(i, j) << 28) | max(i, j)``, so every generated matrix
is symmetric ("draw for i <= j and mirror").

The decay models are the two of the paper's introduction (Sec. I):
exponential |a_ij| < c * lambda^|i-j| and algebraic |a_ij| < c / (|i-j|^l + 1).
The water-cluster-like matrix stands in for the Hilbert-ordered (H2O)_300
RHF/6-31G** density matrix of Sec. IV.B (n = 7500), which is not available:
300 sites uniform in a cube at 0.1 sites per cubic angstrom, ordered along a
3-D Hilbert curve (Skilling 2004), 25 functions per site,
a_ij = g_ij * exp(-0.5 * r_ij) with g_ij ~ N(0, 1).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MAX_INDEX = 1 << 28          # counters hold i, j < 2^28
_CHUNK = 1 << 22              # elements generated per slab


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (xor-shift-multiply finaliser)."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _seed_base(seed: int) -> np.uint64:
    with np.errstate(over="ignore"):
        return _mix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
                      * GAMMA)[0]


def splitmix_u64(seed: int, counters: np.ndarray) -> np.ndarray:
    """64-bit draws for an array of uint64 counters under ``seed``."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _seed_base(seed) + (c + np.uint64(1)) * GAMMA
        return _mix64(z)


def _u01_open_closed(z: np.ndarray) -> np.ndarray:
    """(0, 1] from the top 53 bits."""
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def _uniform_pm1(z: np.ndarray) -> np.ndarray:
    """(-1, 1), symmetric about 0, never +-1."""
    return (((z >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -52)) - 1.0


def pair_counters(stream: int, i: np.ndarray, j: np.ndarray) -> np.ndarray:
    lo = np.minimum(i, j).astype(np.uint64)
    hi = np.maximum(i, j).astype(np.uint64)
    return (np.uint64(stream) << np.uint64(56)) | (lo << np.uint64(28)) | hi


def _row_slabs(n: int):
    rows = max(1, _CHUNK // max(n, 1))
    for r0 in range(0, n, rows):
        yield r0, min(n, r0 + rows)


def _fill(n: int, elem) -> np.ndarray:
    """Assemble an n x n float32 matrix slab by slab; ``elem(i, j)`` gets
    broadcast row/column index grids and returns float64 values."""
    if n <= 0 or n > _MAX_INDEX:
        raise ValueError(f"matrix order {n} out of range")
    out = np.empty((n, n), dtype=np.float32)
    j = np.arange(n, dtype=np.int64)[None, :]
    for r0, r1 in _row_slabs(n):
        i = np.arange(r0, r1, dtype=np.int64)[:, None]
        out[r0:r1] = elem(i, j).astype(np.float32)
    return out


def uniform_pm1(seed: int, stream: int, i, j) -> np.ndarray:
    return _uniform_pm1(splitmix_u64(seed, pair_counters(stream, i, j)))


def normal(seed: int, i, j) -> np.ndarray:
    """N(0, 1) by Box-Muller from streams 1 and 2, symmetric in (i, j)."""
    u1 = _u01_open_closed(splitmix_u64(seed, pair_counters(1, i, j)))
    u2 = _u01_open_closed(splitmix_u64(seed, pair_counters(2, i, j)))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def exp_decay(n: int, lam: float = 0.9, seed: int = 0) -> np.ndarray:
    """a_ij = u_ij * lam^|i-j|, u_ij uniform in (-1, 1), symmetric."""
    loglam = math.log(lam)

    def elem(i, j):
        return uniform_pm1(seed, 0, i, j) * np.exp(loglam * np.abs(i - j))
    return _fill(n, elem)


def algebraic_decay(n: int, seed: int = 0) -> np.ndarray:
    """a_ij = s_ij / (|i-j|^2 + 1) with s_ij = +-1, symmetric."""
    def elem(i, j):
        z = splitmix_u64(seed, pair_counters(3, i, j))
        s = np.where((z >> np.uint64(63)) == 0, 1.0, -1.0)
        d = np.abs(i - j).astype(np.float64)
        return s / (d * d + 1.0)
    return _fill(n, elem)


def uniform_dense(n: int, seed: int = 0, symmetric: bool = True) -> np.ndarray:
    """No decay: a_ij uniform in (-1, 1).  ``symmetric=False`` draws every
    (i, j) independently (stream 4 keyed by the ordered pair)."""
    if symmetric:
        return _fill(n, lambda i, j: uniform_pm1(seed, 0, i, j))

    def elem(i, j):
        c = (np.uint64(4) << np.uint64(56)) | (i.astype(np.uint64) << np.uint64(28)) \
            | j.astype(np.uint64)
        return _uniform_pm1(splitmix_u64(seed, c))
    return _fill(n, elem)


def exp_decay_nonsym(n: int, lam: float = 0.9, seed: int = 0) -> np.ndarray:
    """Exponential decay with independent (i, j) and (j, i) entries; used
    where a test must tell A from its transpose."""
    loglam = math.log(lam)

    def elem(i, j):
        c = (np.uint64(5) << np.uint64(56)) | (i.astype(np.uint64) << np.uint64(28)) \
            | j.astype(np.uint64)
        return _uniform_pm1(splitmix_u64(seed, c)) * np.exp(loglam * np.abs(i - j))
    return _fill(n, elem)


# ---------------------------------------------------------------- Hilbert --

def hilbert_index_3d(coords: np.ndarray, bits: int) -> np.ndarray:
    """Position along a 3-D Hilbert curve of integer coordinates in
    [0, 2^bits), following Skilling's axes-to-transpose construction
    (J. Skilling, AIP Conf. Proc. 707, 381 (2004)): undo the excess work of
    the curve's reflections and exchanges from the top bit down, Gray-encode
    across axes, then interleave the bits of the transposed form."""
    X = [int(v) for v in coords]
    ndim = len(X)
    top = 1 << (bits - 1)
    q = top
    while q > 1:
        p = q - 1
        for a in range(ndim):
            if X[a] & q:
                X[0] ^= p
            else:
                t = (X[0] ^ X[a]) & p
                X[0] ^= t
                X[a] ^= t
        q >>= 1
    for a in range(1, ndim):
        X[a] ^= X[a - 1]
    t = 0
    q = top
    while q > 1:
        if X[ndim - 1] & q:
            t ^= q - 1
        q >>= 1
    for a in range(ndim):
        X[a] ^= t
    h = 0
    for bit in range(bits - 1, -1, -1):
        for a in range(ndim):
            h = (h << 1) | ((X[a] >> bit) & 1)
    return h


def water_like_sites(n_sites: int = 300, density: float = 0.1, seed: int = 0,
                     grid_bits: int = 10):
    """Site positions (angstrom) uniform in a cube holding ``n_sites`` at
    ``density`` sites per cubic angstrom, returned in Hilbert order
    (ties broken by site id)."""
    side = (n_sites / density) ** (1.0 / 3.0)
    ids = np.arange(n_sites, dtype=np.int64)
    pos = np.empty((n_sites, 3))
    for ax in range(3):
        c = (np.uint64(6 + ax) << np.uint64(56)) | ids.astype(np.uint64)
        pos[:, ax] = _u01_open_closed(splitmix_u64(seed, c)) * side
    cells = np.minimum((pos / side * (1 << grid_bits)).astype(np.int64),
                       (1 << grid_bits) - 1)
    keys = [hilbert_index_3d(cells[s], grid_bits) for s in range(n_sites)]
    order = sorted(range(n_sites), key=lambda s: (keys[s], s))
    return pos[order], side


def water_like(n_sites: int = 300, nbf: int = 25, density: float = 0.1,
               seed: int = 0, decay: float = 0.5) -> np.ndarray:
    """Water-cluster-like density matrix stand-in, n = n_sites * nbf:
    a_ij = g_ij * exp(-decay * r_ij[angstrom]), g_ij ~ N(0, 1) symmetric."""
    pos, _ = water_like_sites(n_sites, density, seed)
    n = n_sites * nbf
    site = np.arange(n, dtype=np.int64) // nbf
    diff = pos[:, None, :] - pos[None, :, :]
    rsite = np.sqrt((diff * diff).sum(axis=2))

    def elem(i, j):
        r = rsite[site[i[:, 0]]][:, site[j[0]]]
        return normal(seed, i, j) * np.exp(-decay * r)
    return _fill(n, elem)


# ----------------------------------------------------------- workloads --

def batched_products(count: int = 64, n_lo: int = 512, n_hi: int = 8192,
                     lam_lo: float = 0.8, lam_hi: float = 0.95, seed: int = 0):
    """(n, lambda, seed) of independent exponential-decay products:
    n log-uniform in [n_lo, n_hi], lambda uniform in [lam_lo, lam_hi]."""
    ids = np.arange(count, dtype=np.uint64)
    u_n = _u01_open_closed(splitmix_u64(seed, (np.uint64(9) << np.uint64(56)) | ids))
    u_l = _u01_open_closed(splitmix_u64(seed, (np.uint64(10) << np.uint64(56)) | ids))
    ns = np.exp(math.log(n_lo) + u_n * (math.log(n_hi) - math.log(n_lo)))
    lams = lam_lo + u_l * (lam_hi - lam_lo)
    return [(int(min(n_hi, max(n_lo, round(x)))), float(l), int(seed * 1000 + k + 1))
            for k, (x, l) in enumerate(zip(ns, lams))]


def poisson_arrivals(count: int, rate: float, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson process with ``rate`` per second."""
    ids = np.arange(count, dtype=np.uint64)
    u = _u01_open_closed(splitmix_u64(seed, (np.uint64(11) << np.uint64(56)) | ids))
    return np.cumsum(-np.log(u) / rate)


def serving_requests(count: int = 64, rate: float = 200.0, n_lo: int = 1024,
                     n_hi: int = 32768, taus=(1e-6, 1e-8), seed: int = 0):
    """Request stream: (arrival_s, n, tau, seed) with n log-uniform."""
    t = poisson_arrivals(count, rate, seed)
    ids = np.arange(count, dtype=np.uint64)
    u_n = _u01_open_closed(splitmix_u64(seed, (np.uint64(12) << np.uint64(56)) | ids))
    z_t = splitmix_u64(seed, (np.uint64(13) << np.uint64(56)) | ids)
    ns = np.exp(math.log(n_lo) + u_n * (math.log(n_hi) - math.log(n_lo)))
    out = []
    for k in range(count):
        n = int(min(n_hi, max(n_lo, round(ns[k]))))
        tau = taus[int(z_t[k] % np.uint64(len(taus)))]
        out.append((float(t[k]), n, float(tau), int(seed * 1000 + k + 1)))
    return out
