"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle,
element by element on the same seeded inputs.

Bars: the surviving-triple set is bit-exact apart from triples whose norm
product is within 1e-6 relative of tau; C agrees with the oracle within
max|dC| / max|C| <= 1e-5 for FP32 and 3xTF32 leaf products; squared norms
agree to 1e-12 relative (FP64 sums in a different order)."""
import math

import numpy as np
import pytest

import spamm_inputs as gen
from oracle import oracle as O
from tests.spamm_check import (as_set, blocks_from, compare_triples, rel_max_err,
                               sample_blocks)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "tf32x3": 1e-5, "bf16x3": 1e-4, "tf32": 2e-3}


def _spamm():
    import paper_1203_1692_gb300 as P
    return P


def _dev(A, lda=None):
    n = A.shape[0]
    if lda is None or lda == n:
        return torch.from_numpy(np.ascontiguousarray(A)).cuda()
    buf = torch.full((n, lda), float("nan"), dtype=torch.float32, device="cuda")
    buf[:, :n] = torch.from_numpy(A).cuda()
    return buf[:, :n]


def _run(A, B, b, tau, precision="fp32", alpha=1.0, beta=0.0, C0=None, lda=None, **kw):
    P = _spamm()
    ctx = P.Context(leaf=b, precision=precision, **kw)
    dA = _dev(A, lda)
    ta = ctx.build_norms(dA)
    if B is A:
        tb, dB = ta, dA
    else:
        dB = _dev(B, lda)
        tb = ctx.build_norms(dB)
    C = torch.from_numpy(np.ascontiguousarray(C0)).cuda() if C0 is not None else None
    C = ctx.multiply(ta, tb, tau, alpha, beta, C)
    torch.cuda.synchronize()
    return ctx, ta, tb, C.cpu().numpy()


# ----------------------------------------------------------------- norms

@pytest.mark.parametrize("n,b,lda", [(64, 16, None), (100, 16, None), (1000, 16, None),
                                     (257, 32, None), (300, 64, 301), (130, 16, 135),
                                     (1, 16, None), (16, 16, None), (17, 16, None),
                                     (500, 128, 512)])
def test_norm_pyramid_matches_oracle(n, b, lda):
    A = gen.exp_decay_nonsym(n, 0.85, seed=n)
    P = _spamm()
    ctx = P.Context(leaf=b)
    t = ctx.build_norms(_dev(A, lda))
    got = t.norms()
    ref = O.pyramid(A, b)
    assert t.depth == O.depth(n, b)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("b", [16, 32, 64, 128])
def test_norms_of_wide_range_and_subnormal_entries(b):
    """Leaf squares are exact and their sums stay within 1e-12 of FP64
    whatever the magnitudes: entries spread over 1e-40 .. 1e30, a block of
    subnormals, a block near FP32's largest values, exact zeros."""
    n = 300
    rng = np.random.default_rng(b)
    A = gen.uniform_dense(n, seed=b, symmetric=False).astype(np.float64)
    A *= 10.0 ** rng.uniform(-40, 30, size=(n, n))
    A[:40, :40] = gen.uniform_dense(40, seed=1).astype(np.float64) * 1e-42
    A[100:140, 200:240] = gen.uniform_dense(40, seed=2).astype(np.float64) * 1e18
    A[250:, :50] = 0.0
    A = A.astype(np.float32)
    ctx = _spamm().Context(leaf=b)
    got = ctx.build_norms(_dev(A)).norms()
    ref = O.pyramid(A, b)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
    assert np.array_equal(got == 0, ref == 0)


# ---------------------------------------------------- triples and C, FP32

CASES = [  # n, b, generator, tau
    (1024, 16, "exp", 1e-6),       # the n = 1024 exponential-decay workload
    (1000, 16, "exp", 1e-4),       # ragged: 1000 = 62.5 leaves
    (700, 32, "water", 1e-3),
    (515, 16, "alg", 1e-5),
    (384, 64, "exp", 1e-2),
    (256, 128, "exp", 1e-1),
    (333, 16, "dense", 0.0),       # tau = 0: the full dense product
]


def _matrix(kind, n, seed=0):
    if kind == "exp":
        return gen.exp_decay(n, 0.9, seed=seed)
    if kind == "alg":
        return gen.algebraic_decay(n, seed=seed)
    if kind == "water":
        return gen.water_like(n // 25, 25, seed=seed) if n % 25 == 0 else gen.exp_decay(n)
    return gen.uniform_dense(n, seed=seed, symmetric=False)


@pytest.mark.parametrize("n,b,kind,tau", CASES)
def test_fp32_parity_with_oracle(n, b, kind, tau):
    A = _matrix(kind, n)
    B = _matrix("exp", n, seed=1) if kind == "dense" else A
    ctx, ta, tb, C = _run(A, B, b, tau)
    ref = O.multiply(A, B, b, tau)
    st = ctx.stats()
    d = O.depth(n, b)
    pa, pb = O.pyramid(A, b), O.pyramid(B, b)
    ndiff = compare_triples(ctx.triples(), ref.triples, pa, pb, d, tau)
    if ndiff == 0:
        assert st["tier_kept"] == list(ref.kept)
        assert st["tier_candidates"] == list(ref.cand)
    assert rel_max_err(C, ref.C) <= TOL["fp32"]
    assert st["leaf_triples"] == len(ctx.triples())
    assert st["kept_flops"] == 2.0 * b ** 3 * st["leaf_triples"]


def test_nonsymmetric_operands_not_transposed():
    n, b = 300, 16
    A = gen.exp_decay_nonsym(n, 0.9, seed=3)
    B = gen.uniform_dense(n, seed=4, symmetric=False)
    ctx, _, _, C = _run(A, B, b, 1e-3)
    ref = O.multiply(A, B, b, 1e-3)
    assert rel_max_err(C, ref.C) <= 1e-5
    assert as_set(ctx.triples()) == as_set(ref.triples)


def test_alpha_beta_and_unread_C():
    n, b = 200, 16
    A = gen.exp_decay(n, 0.8, seed=1)
    C0 = gen.uniform_dense(n, seed=9, symmetric=False)
    _, _, _, C = _run(A, A, b, 1e-4, alpha=-1.5, beta=0.25, C0=C0)
    ref = O.multiply(A, A, b, 1e-4, alpha=-1.5, beta=0.25, C=C0.astype(np.float64))
    assert rel_max_err(C, ref.C) <= 1e-5
    Cnan = np.full((n, n), np.nan, dtype=np.float32)
    _, _, _, C2 = _run(A, A, b, 1e-4, alpha=1.0, beta=0.0, C0=Cnan)
    assert np.isfinite(C2).all()


def test_tau_above_root_gives_beta_C():
    n, b = 128, 16
    A = gen.exp_decay(n, 0.9, seed=2)
    root = float(np.linalg.norm(A.astype(np.float64))) ** 2
    C0 = gen.uniform_dense(n, seed=5, symmetric=False)
    ctx, _, _, C = _run(A, A, b, root * 1.001, alpha=1.0, beta=0.5, C0=C0)
    assert ctx.stats()["leaf_triples"] == 0
    np.testing.assert_array_equal(C, (0.5 * C0).astype(np.float32))


def test_deterministic_bitwise():
    n, b = 1024, 16
    A = gen.exp_decay(n, 0.9)
    _, _, _, C1 = _run(A, A, b, 1e-6)
    _, _, _, C2 = _run(A, A, b, 1e-6)
    np.testing.assert_array_equal(C1, C2)


def test_nonfinite_input_is_reported():
    P = _spamm()
    n = 64
    A = gen.exp_decay(n, 0.9)
    A[10, 20] = np.nan
    ctx = P.Context(leaf=16)
    t = ctx.build_norms(_dev(A))
    with pytest.raises(P.SpammError, match="NONFINITE"):
        ctx.multiply(t, t, 1e-6)


def test_invalid_arguments():
    P = _spamm()
    ctx = P.Context(leaf=16)
    A = _dev(gen.exp_decay(64, 0.9))
    t = ctx.build_norms(A)
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(P.SpammError, match="INVALID_ARG"):
            ctx.multiply(t, t, bad)
    ctx2 = P.Context(leaf=32)
    t2 = ctx2.build_norms(A)
    with pytest.raises(P.SpammError, match="INVALID_ARG"):
        ctx.multiply(t, t2, 1e-3)


def test_pool_overflow_checked_and_unchecked():
    P = _spamm()
    n, b = 1024, 16
    A = gen.uniform_dense(n, seed=1)
    dA = _dev(A)
    ref = O.multiply(A, A, b, 0.0)
    # unchecked: tiny pool -> CAPACITY through stats, C untouched
    ctx = P.Context(leaf=b, pool_bytes=16384, checked=False)
    t = ctx.build_norms(dA)
    C = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    ctx.multiply(t, t, 0.0, C=C)
    with pytest.raises(P.SpammError, match="CAPACITY"):
        ctx.stats()
    need = ctx.stats(raise_on_error=False)["pool_needed_bytes"]
    assert need > 16384
    assert not C.any()
    # checked: grows the pool and re-runs
    ctx2 = P.Context(leaf=b, pool_bytes=16384, checked=True)
    t2 = ctx2.build_norms(dA)
    C2 = ctx2.multiply(t2, t2, 0.0)
    assert rel_max_err(C2.cpu().numpy(), ref.C) <= 1e-5
    assert ctx2.stats()["leaf_triples"] == (n // b) ** 3


@pytest.mark.parametrize("n", [1, 5, 16, 17, 31, 129])
def test_tiny_and_ragged_sizes(n):
    A = gen.uniform_dense(n, seed=n, symmetric=False)
    for b in (16, 32):
        ctx, _, _, C = _run(A, A, b, 0.0)
        ref = O.multiply(A, A, b, 0.0)
        assert rel_max_err(C, ref.C) <= 1e-5
        assert as_set(ctx.triples()) == as_set(ref.triples)


def test_host_entry_point_matches_device_entry_point():
    P = _spamm()
    n, b = 640, 16
    A = gen.exp_decay(n, 0.9, seed=7)
    ctx = P.Context(leaf=b)
    Ch = ctx.multiply_host(A, None, 1e-5)
    _, _, _, Cd = _run(A, A, b, 1e-5)
    np.testing.assert_array_equal(Ch, Cd)


# ------------------------------------------------ full-size, sampled blocks

def _sampled_parity(A, b, tau, precision, count=24):
    n = A.shape[0]
    ctx, ta, tb, C = _run(A, A, b, tau, precision=precision)
    ij = sample_blocks(n, b, count)
    pa = O.pyramid(A, b)
    ref, _ = O.blocks(A, A, b, tau, ij, pa, pa)
    got = blocks_from(C, ij, b, n)
    err = float(np.abs(got - ref).max() / np.abs(ref).max())
    # triple counts: the oracle's flat count over the sampled blocks
    return ctx, err


@pytest.mark.slow
def test_water_like_n7500_sampled():
    A = gen.water_like()
    ctx, err = _sampled_parity(A, 16, 1e-6, "fp32")
    assert err <= 1e-5
    st = ctx.stats()
    assert st["depth"] == 9 and st["leaf_triples"] > 0


def test_tree_outliving_its_context_is_freed_safely():
    """A tree freed after its context (as garbage collection may order it)
    must not touch the freed context."""
    P = _spamm()
    for prec in ("fp32", "tf32x3"):
        ctx = P.Context(leaf=16, precision=prec)
        A = _dev(gen.exp_decay(300, 0.9, seed=1))
        t = ctx.build_norms(A)
        ctx.multiply(t, t, 1e-6)
        ctx.close()
        t.close()


FLAT_CASES = [(1024, 16, "exp", 1e-6), (700, 32, "water", 1e-3), (515, 16, "alg", 1e-5),
              (333, 16, "dense", 0.0), (1000, 64, "exp", 1e-4), (17, 16, "exp", 1e-3)]


@pytest.mark.parametrize("n,b,kind,tau", FLAT_CASES)
def test_flat_enumeration_equals_hierarchy_and_oracle(n, b, kind, tau):
    """Algorithm 1's flat, norm-sorted enumeration on the GPU keeps exactly
    the leaf triples of the tier-by-tier cull (same leaf test, parent norms
    never below their children's), and the oracle's outside the tie band."""
    A = _matrix(kind, n)
    B = _matrix("exp", n, seed=1) if kind == "dense" else A
    P = _spamm()
    ctx = P.Context(leaf=b, precision="fp32")
    ta = ctx.build_norms(_dev(A))
    tb = ctx.build_norms(_dev(B))
    ctx.multiply(ta, tb, tau)
    hier = ctx.triples()
    flat, cnt, ms = ctx.cull_flat(ta, tb, tau)
    assert cnt == len(flat) == len(hier)
    assert as_set(flat) == as_set(hier)
    _, cnt_only, _ = ctx.cull_flat(ta, tb, tau, triples=False)
    assert cnt_only == cnt
    ref = O.multiply(A, B, b, tau)
    compare_triples(flat, ref.triples, O.pyramid(A, b), O.pyramid(B, b), O.depth(n, b), tau)
    linkless = O.cull_linkless(O.pyramid(A, b), O.pyramid(B, b), O.depth(n, b), tau)
    if ctx.stats()["tie_band"] == 0:
        assert as_set(flat) == as_set(linkless)
