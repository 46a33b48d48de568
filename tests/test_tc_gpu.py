"""Parity of the tcgen05 leaf kernel with the FP64 oracle, through the C ABI.

The symbolic stages are shared with the FP32 path, so the surviving-triple
set must match the oracle exactly as there.  Tolerances on
max|dC| / max|C| follow from each precision's operand splitting:
  tf32x3  a = hi + lo + r with |r| <= 2^-22 |a|; dropped lo*lo and r terms
          give ~3 * 2^-22 = 7e-7 per product, plus FP32 accumulation -> 1e-5
          (the FP32 bar);
  bf16x3  |r| <= 2^-18 |a|, ~3 * 2^-18 = 1.1e-5 per product, times a
          condition sum |a||b| / max|C| of a few -> 1e-4;
  tf32    one pass, |a - hi| <= 2^-11 |a| per operand, ~2^-10 per product
          -> 5e-3.
"""
import numpy as np
import pytest

import spamm_inputs as gen
from oracle import oracle as O
from tests.spamm_check import (as_set, blocks_from, compare_triples, compare_triples_large,
                               rel_max_err,
                               sample_blocks)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"tf32x3": 1e-5, "f16x3": 1e-5, "bf16x3": 1e-4, "tf32": 5e-3}


def _run(A, B, b, tau, precision, alpha=1.0, beta=0.0, C0=None):
    import paper_1203_1692_gb300 as P
    ctx = P.Context(leaf=b, precision=precision)
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    ta = ctx.build_norms(dA)
    if B is A:
        tb = ta
    else:
        dB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
        tb = ctx.build_norms(dB)
    C = torch.from_numpy(np.ascontiguousarray(C0)).cuda() if C0 is not None else None
    C = ctx.multiply(ta, tb, tau, alpha, beta, C)
    torch.cuda.synchronize()
    return ctx, C.cpu().numpy()


def _matrix(kind, n, seed=0):
    if kind == "exp":
        return gen.exp_decay(n, 0.9, seed=seed)
    if kind == "alg":
        return gen.algebraic_decay(n, seed=seed)
    if kind == "water":
        return gen.water_like(n // 25, 25, seed=seed)
    return gen.uniform_dense(n, seed=seed, symmetric=False)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "tf32"])
def test_single_tile(prec):
    n, b = 128, 16
    A = _matrix("exp", n)
    ctx, C = _run(A, A, b, 1e-6, prec)
    ref = O.multiply(A, A, b, 1e-6)
    assert as_set(ctx.triples()) == as_set(ref.triples)
    assert rel_max_err(C, ref.C) <= TOL[prec]


CASES = [
    (1024, 16, "exp", 1e-6),
    (1000, 16, "exp", 1e-4),
    (700, 32, "water", 1e-3),
    (515, 16, "alg", 1e-5),
    (333, 16, "dense", 0.0),
    (333, 32, "dense", 0.0),
    (600, 32, "exp", 1e-5),
    (640, 64, "exp", 1e-5),
    (530, 64, "alg", 1e-6),        # ragged: 530 = 8.3 leaves of 64
    (300, 64, "dense", 0.0),
    (768, 128, "exp", 1e-6),
    (450, 128, "alg", 1e-5),       # ragged, one pair tile of 128-leaves
]


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "tf32", "f16x3"])
@pytest.mark.parametrize("n,b,kind,tau", CASES)
def test_tc_parity_with_oracle(prec, n, b, kind, tau):
    A = _matrix(kind, n)
    B = _matrix("exp", n, seed=1) if kind == "dense" else A
    ctx, C = _run(A, B, b, tau, prec)
    ref = O.multiply(A, B, b, tau)
    d = O.depth(n, b)
    compare_triples(ctx.triples(), ref.triples, O.pyramid(A, b), O.pyramid(B, b), d, tau)
    assert rel_max_err(C, ref.C) <= TOL[prec]
    # kept flops over each leaf's extent inside the matrix (Appendix A's 2 m n k
    # per product, the zero padding of the ragged last leaves left out)
    st = ctx.stats()
    if st["tie_band"] == 0:
        ext = lambda L: np.minimum(b, n - np.asarray(L, dtype=np.int64) * b)
        t = ref.triples
        want = 2.0 * float(np.sum(ext(t[:, 0]) * ext(t[:, 1]) * ext(t[:, 2])))
        assert st["kept_flops_clipped"] == want
        assert st["kept_flops_clipped"] <= st["kept_flops"]


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "f16x3"])
def test_tc_alpha_beta(prec):
    n, b = 260, 16
    A = gen.exp_decay_nonsym(n, 0.85, seed=2)
    B = gen.exp_decay_nonsym(n, 0.85, seed=3)
    C0 = gen.uniform_dense(n, seed=4, symmetric=False)
    _, C = _run(A, B, b, 1e-4, prec, alpha=0.5, beta=-2.0, C0=C0)
    ref = O.multiply(A, B, b, 1e-4, alpha=0.5, beta=-2.0, C=C0.astype(np.float64))
    assert rel_max_err(C, ref.C) <= TOL[prec]


def test_tc_deterministic():
    A = _matrix("exp", 1024)
    _, C1 = _run(A, A, 16, 1e-6, "tf32x3")
    _, C2 = _run(A, A, 16, 1e-6, "tf32x3")
    np.testing.assert_array_equal(C1, C2)


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_tc_water_like_n7500_sampled(prec):
    A = gen.water_like()
    n, b, tau = A.shape[0], 16, 1e-6
    ctx, C = _run(A, A, b, tau, prec)
    ij = sample_blocks(n, b, 24)
    pa = O.pyramid(A, b)
    ref, _ = O.blocks(A, A, b, tau, ij, pa, pa)
    got = blocks_from(C, ij, b, n)
    assert float(np.abs(got - ref).max() / np.abs(ref).max()) <= TOL[prec]


@pytest.mark.slow
@pytest.mark.parametrize("prec,b", [("tf32x3", 64), ("bf16x3", 64), ("f16x3", 64),
                                    ("f16x3", 128), ("tf32x3", 128)])
def test_tc_water_like_n7500_bench_configuration(prec, b):
    """The bench's launch configurations on the n = 7500 workload (leaf 64
    and leaf 128, which the bench's leaf trials pick between, at tau 1e-4):
    the whole surviving-triple set against the oracle's flat enumeration
    (Algorithm 1) bit for bit outside the tie band, the per-tier counts
    against the oracle's recursion, and sampled C blocks against the
    oracle."""
    A = gen.water_like()
    n, tau = A.shape[0], 1e-4
    ctx, C = _run(A, A, b, tau, prec)
    pa = O.pyramid(A, b)
    d = O.depth(n, b)
    st = ctx.stats()
    flat = O.cull_linkless(pa, pa, d, tau)
    ndiff = compare_triples_large(ctx.triples(), flat, pa, pa, d, tau)
    assert ndiff <= st["tie_band"]
    _, cand, kept = O.cull_recursive(pa, pa, d, tau)
    if st["tie_band"] == 0:
        assert st["tier_kept"] == kept.tolist()
        assert st["tier_candidates"] == cand.tolist()
    ij = sample_blocks(n, b, 24)
    ref, _ = O.blocks(A, A, b, tau, ij, pa, pa)
    got = blocks_from(C, ij, b, n)
    assert float(np.abs(got - ref).max() / np.abs(ref).max()) <= TOL[prec]


@pytest.mark.slow
@pytest.mark.parametrize("prec,b", [("tf32x3", 16), ("bf16x3", 16), ("tf32", 16),
                                    ("tf32x3", 64), ("f16x3", 64)])
def test_tc_algebraic_n16384_sampled(prec, b):
    """The algebraic-decay configuration at full size (n = 16384, tau =
    1e-8, leaf products in TF32, split BF16 x3 and 3xTF32): sampled C blocks
    against the oracle, and the whole surviving-triple set against the
    oracle's flat enumeration (|s_ij| = 1, so every leaf norm, and hence the
    set, is sign-free)."""
    A = gen.algebraic_decay(16384, seed=0)
    n, tau = A.shape[0], 1e-8
    ctx, C = _run(A, A, b, tau, prec)
    ij = sample_blocks(n, b, 16)
    pa = O.pyramid(A, b)
    ref, _ = O.blocks(A, A, b, tau, ij, pa, pa)
    got = blocks_from(C, ij, b, n)
    assert float(np.abs(got - ref).max() / np.abs(ref).max()) <= TOL[prec]
    # the whole surviving-triple set against the oracle's flat enumeration
    # on the same norms (bit for bit outside the tie band)
    d = O.depth(n, b)
    flat = O.cull_linkless(pa, pa, d, tau)
    st = ctx.stats()
    ndiff = compare_triples_large(ctx.triples(), flat, pa, pa, d, tau)
    assert ndiff <= st["tie_band"]
    if st["tie_band"] == 0:
        assert st["leaf_triples"] == len(flat)


@pytest.mark.parametrize("prec,b", [("tf32x3", 16), ("bf16x3", 32), ("tf32x3", 64),
                                    ("f16x3", 64)])
def test_tc_stale_pieces_never_reach_C(prec, b):
    """A multiply packs only the leaves that can take part in a kept product
    (Sec. III culling is monotone in each norm).  Pieces it does not pack
    keep whatever an earlier multiply left there; here that is a matrix of
    1e15s packed in full at tau = 0, and none of it may leak into C."""
    import paper_1203_1692_gb300 as P
    n = 700
    ctx = P.Context(leaf=b, precision=prec)
    big = torch.full((n, n), 1e15, dtype=torch.float32, device="cuda")
    tree = ctx.build_norms(big)
    C = torch.empty_like(big)
    ctx.multiply(tree, tree, 0.0, C=C)
    A = _matrix("exp", n)
    dA = torch.from_numpy(A).cuda()
    tree.rebuild(dA)
    for tau in (1e-2, 1e-5):
        ctx.multiply(tree, tree, tau, C=C)
        ref = O.multiply(A, A, b, tau)
        assert rel_max_err(C.cpu().numpy(), ref.C) <= TOL[prec]
    # another right operand through the same left tree
    Bm = gen.exp_decay_nonsym(n, 0.85, seed=9)
    tb = ctx.build_norms(torch.from_numpy(Bm).cuda())
    ctx.multiply(tree, tb, 1e-4, C=C)
    ref = O.multiply(A, Bm, b, 1e-4)
    assert rel_max_err(C.cpu().numpy(), ref.C) <= TOL[prec]


SLICE_CASES = [
    (640, 64, "exp", 1e-5),
    (530, 32, "alg", 1e-6),        # ragged
    (450, 128, "exp", 1e-4),
    (300, 64, "dense", 0.0),       # tau = 0: every non-zero panel kept
    (1000, 64, "water", 1e-3),
]


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "f16x3"])
@pytest.mark.parametrize("n,b,kind,tau", SLICE_CASES)
def test_slice_cull_parity_with_oracle(prec, n, b, kind, tau):
    """Sub-leaf cull along k (16-wide slices of each kept leaf product,
    the paper's SpAMM(4x4) read for tensor cores) against the oracle's
    sliced product: C within the precision's tolerance, the same leaf
    triples and the same number of kept slice products outside ties."""
    import paper_1203_1692_gb300 as P
    A = _matrix(kind, n)
    B = _matrix("exp", n, seed=1) if kind == "dense" else A
    ctx = P.Context(leaf=b, precision=prec, slice=16)
    ta = ctx.build_norms(torch.from_numpy(A).cuda())
    tb = ta if B is A else ctx.build_norms(torch.from_numpy(B).cuda())
    C = ctx.multiply(ta, tb, tau)
    torch.cuda.synchronize()
    st = ctx.stats()
    refC, m, kept, tested = O.multiply_sliced(A, B, b, 16, tau)
    assert rel_max_err(C.cpu().numpy(), refC) <= TOL[prec]
    if st["tie_band"] == 0:
        assert st["leaf_triples"] == m
        assert st["slice_tested"] == tested and st["slice_kept"] == kept
    else:
        assert abs(st["slice_kept"] - kept) <= st["tie_band"]
    assert st["kept_flops"] == 2.0 * b * b * 16 * st["slice_kept"]


def test_slice_cull_matches_plain_when_nothing_is_culled_inside_leaves():
    """At tau = 0 every slice with two non-zero panels is kept, so the
    sliced product equals the plain one (same accumulation order)."""
    import paper_1203_1692_gb300 as P
    A = _matrix("exp", 512)
    dA = torch.from_numpy(A).cuda()
    out = []
    for sl in (0, 16):
        ctx = P.Context(leaf=64, precision="tf32x3", slice=sl)
        t = ctx.build_norms(dA)
        out.append(ctx.multiply(t, t, 0.0).cpu().numpy())
    np.testing.assert_array_equal(out[0], out[1])


def test_slice_cull_batched_equals_single():
    import paper_1203_1692_gb300 as P
    mats = [_matrix("exp", n, seed=n) for n in (300, 700, 1000)]
    ctx = P.Context(leaf=64, precision="tf32x3", slice=16)
    dm = [torch.from_numpy(A).cuda() for A in mats]
    trees = [ctx.build_norms(A) for A in dm]
    Cs = ctx.multiply_batched(trees, trees, [1e-5, 1e-4, 1e-6])
    for A, t, C, tau in zip(dm, trees, Cs, [1e-5, 1e-4, 1e-6]):
        c1 = P.Context(leaf=64, precision="tf32x3", slice=16)
        t1 = c1.build_norms(A)
        assert torch.equal(c1.multiply(t1, t1, tau), C)


def test_f16x3_wide_dynamic_range():
    """The FP16 split scales each operand by a power of two so its largest
    leaf norm sits just below 2^15; entries many decades smaller (down to
    fp16 subnormals after scaling) still reach 3xTF32-class accuracy in the
    max-norm."""
    n, b, tau = 600, 32, 0.0
    rng = np.random.default_rng(3)
    A = (gen.uniform_dense(n, seed=1, symmetric=False).astype(np.float64)
         * 10.0 ** rng.uniform(-12, 6, size=(n, n))).astype(np.float32)
    B = (gen.uniform_dense(n, seed=2, symmetric=False).astype(np.float64) * 1e-20).astype(np.float32)
    ref = O.multiply(A, B, b, tau)
    for prec in ("f16x3", "tf32x3"):
        _, C = _run(A, B, b, tau, prec)
        assert rel_max_err(C, ref.C) <= TOL[prec], prec


@pytest.mark.parametrize("sa,sb", [(110, -120), (-120, 100), (-50, -45)])
def test_f16x3_extreme_operand_scales(sa, sb):
    """Operands near the ends of the float range: the power-of-two scales
    (one per operand, up to 2^126 each way) keep every split inside fp16's
    range, and the unscale 2^-(kA + kB), which can lie outside one float's
    exponent range, is applied as two exact factors."""
    n, b, tau = 520, 32, 0.0
    A = (gen.uniform_dense(n, seed=5, symmetric=False).astype(np.float64) * 2.0 ** sa).astype(np.float32)
    B = (gen.uniform_dense(n, seed=6, symmetric=False).astype(np.float64) * 2.0 ** sb).astype(np.float32)
    assert np.isfinite(A).all() and np.isfinite(B).all() and np.abs(B).max() > 2.0 ** -126
    ref = O.multiply(A, B, b, tau)
    assert np.abs(ref.C).max() > 2.0 ** -100          # a normal-range product
    _, C = _run(A, B, b, tau, "f16x3")
    assert np.isfinite(C).all()
    assert rel_max_err(C, ref.C) <= TOL["f16x3"]


@pytest.mark.parametrize("prec,b,n,pinned", [("f16x3", 64, 2600, True), ("tf32x3", 32, 1500, False),
                                             ("f16x3", 16, 700, True), ("bf16x3", 128, 300, False),
                                             ("tf32", 64, 5000, True)])
def test_host_entry_bands_equal_device_multiply(prec, b, n, pinned):
    """The host entry point runs the leaf products in (up to) three launches
    of whole tile-row groups and copies each group's rows of C out while the
    next computes.  C is the device multiply's, bit for bit, with alpha and
    beta, from pageable and from pinned host memory."""
    import paper_1203_1692_gb300 as P
    A = gen.exp_decay(n, 0.9, seed=3)
    B = gen.uniform_dense(n, seed=4, symmetric=False)
    C0 = gen.uniform_dense(n, seed=5, symmetric=False)
    tau, alpha, beta = 1e-5, 0.75, -0.5
    _, Cd = _run(A, B, b, tau, prec, alpha, beta, C0)
    ctx = P.Context(leaf=b, precision=prec)
    if pinned:
        Ah = torch.from_numpy(A).pin_memory()
        Bh = torch.from_numpy(B).pin_memory()
        Ch = torch.from_numpy(C0.copy()).pin_memory()
        ctx.multiply_host(Ah, Bh, tau, alpha, beta, C=Ch)
        Ch = Ch.numpy()
    else:
        Ch = C0.copy()
        ctx.multiply_host(A, B, tau, alpha, beta, C=Ch)
    assert np.array_equal(Ch, Cd)
    # and again on the same context (staging and trees reused)
    Ch2 = C0.copy()
    ctx.multiply_host(A, B, tau, alpha, beta, C=Ch2)
    assert np.array_equal(Ch2, Cd)


@pytest.mark.parametrize("prec,b", [("f16x3", 32), ("tf32x3", 64)])
def test_packed_leaf_counts(prec, b):
    """stats() counts the leaves the packs hold: leaf (I, K) in the A role
    iff ||A_IK||^2 max_J ||B_KJ||^2 passes the SpAMM test, leaf (K, J) in the
    B role iff max_I ||A_IK||^2 ||B_KJ||^2 does (the monotone bound that
    decides which pieces a kept product can read); recounted here from the
    oracle's leaf norms."""
    n, tau = 1200, 1e-3
    A = gen.exp_decay(n, 0.8, seed=1)
    B = gen.exp_decay(n, 0.85, seed=2)
    ctx, _ = _run(A, B, b, tau, prec)
    st = ctx.stats()
    d = O.depth(n, b)
    la = O.tier(O.pyramid(A, b), d)
    lb = O.tier(O.pyramid(B, b), d)
    nl = -(-n // b)
    la, lb = la[:nl, :nl], lb[:nl, :nl]
    rowmaxB = lb.max(axis=1)            # per K: max_J ||B_KJ||^2
    colmaxA = la.max(axis=0)            # per K: max_I ||A_IK||^2
    pa = la * rowmaxB[None, :]
    pb = colmaxA[:, None] * lb
    t2 = tau * tau
    # no product near the threshold, so the exact test and this one agree
    for p in (pa, pb):
        assert np.all(np.abs(p[p > 0] - t2) > 1e-6 * t2)
    want_a = int(np.count_nonzero((pa >= t2) & (la > 0) & (rowmaxB[None, :] > 0)))
    want_b = int(np.count_nonzero((pb >= t2) & (lb > 0) & (colmaxA[:, None] > 0)))
    assert 0 < want_a < nl * nl and 0 < want_b < nl * nl
    assert st["packed_leaves_a"] == want_a
    assert st["packed_leaves_b"] == want_b
    # a dense product packs every leaf in both roles
    D = gen.uniform_dense(n, seed=3, symmetric=False)
    ctx2, _ = _run(D, D, b, 0.0, prec)
    st2 = ctx2.stats()
    assert st2["packed_leaves_a"] == nl * nl and st2["packed_leaves_b"] == nl * nl
