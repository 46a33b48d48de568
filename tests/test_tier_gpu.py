"""Precision chosen by norm (reading R16, config tier_bits) on the tensor
cores, through the C ABI, against the FP64 oracle's tiered product.

The SpAMM condition (Eq. (norm_condition)) is applied a second time, at
tau_h = 2^tier_bits tau: a kept leaf product with ||A_IK|| ||B_KJ|| >= tau_h
keeps the full split (three passes), the others run one pass on the high
parts.  The oracle forms the one-pass products from operands rounded to the
high part's significant bits (11 for f16x3 and tf32x3, 8 for bf16x3), so the
GPU and the oracle differ only by the tensor core's FP32 accumulation and
the same tolerances as the plain split products apply.  The kept set and
the full-split subset must both match the oracle bit for bit outside their
tie bands (around tau and tau_h)."""
import numpy as np
import pytest

import spamm_inputs as gen
from oracle import oracle as O
from tests.spamm_check import (blocks_from, compare_triples, compare_triples_large,
                               rel_max_err, sample_blocks)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"tf32x3": 1e-5, "f16x3": 1e-5, "bf16x3": 1e-4}


def _matrix(kind, n, seed=0):
    if kind == "exp":
        return gen.exp_decay(n, 0.9, seed=seed)
    if kind == "alg":
        return gen.algebraic_decay(n, seed=seed)
    if kind == "water":
        return gen.water_like(n // 25, 25, seed=seed)
    if kind == "nonsym":
        return gen.exp_decay_nonsym(n, 0.85, seed=seed)
    return gen.uniform_dense(n, seed=seed, symmetric=False)


def _hi_set(A, B, b, tau_h, triples):
    """Kept triples whose oracle norm product reaches tau_h."""
    d = O.depth(A.shape[0], b)
    la = O.tier(O.pyramid(A, b), d)
    lb = O.tier(O.pyramid(B, b), d)
    t = np.asarray(triples).reshape(-1, 3)
    p = la[t[:, 0], t[:, 1]] * lb[t[:, 1], t[:, 2]]
    return t[p >= tau_h * tau_h]


def _run(A, B, b, tau, prec, bits, alpha=1.0, beta=0.0, C0=None, slice=0):
    import paper_1203_1692_gb300 as P
    ctx = P.Context(leaf=b, precision=prec, tier_bits=bits, slice=slice)
    ta = ctx.build_norms(torch.from_numpy(np.ascontiguousarray(A)).cuda())
    tb = ta if B is A else ctx.build_norms(torch.from_numpy(np.ascontiguousarray(B)).cuda())
    C = torch.from_numpy(np.ascontiguousarray(C0)).cuda() if C0 is not None else None
    C = ctx.multiply(ta, tb, tau, alpha, beta, C)
    torch.cuda.synchronize()
    return ctx, C.cpu().numpy()


CASES = [
    (1024, 16, "exp", 1e-6),
    (1000, 16, "nonsym", 1e-4),
    (700, 32, "water", 1e-3),
    (515, 16, "alg", 1e-5),
    (600, 32, "exp", 1e-5),
    (640, 64, "exp", 1e-5),
    (530, 64, "alg", 1e-6),        # ragged: 530 = 8.3 leaves of 64
    (1000, 64, "water", 1e-3),
    (768, 128, "exp", 1e-6),
    (450, 128, "alg", 1e-5),       # ragged, one pair tile of 128-leaves
]


@pytest.mark.parametrize("prec", ["f16x3", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("shift", [0, 4])
@pytest.mark.parametrize("n,b,kind,tau", CASES)
def test_tier_parity_with_oracle(prec, shift, n, b, kind, tau):
    """tier_bits = p - 1 (each one-pass product errs by about tau) and
    p + 3 (sixteen times more): C against the oracle's tiered product, the
    kept set and the full-split set against the oracle's."""
    p, away = O.HIGH_PART[prec]
    bits = p - 1 + shift
    tau_h = tau * 2.0 ** bits
    A = _matrix(kind, n)
    B = A if kind in ("exp", "water", "alg") else _matrix("exp", n, seed=1)
    ctx, C = _run(A, B, b, tau, prec, bits)
    refC, m, exact, rounded = O.multiply_tiered(A, B, b, tau, tau_h, p, away)
    st = ctx.stats()
    d = O.depth(n, b)
    pa, pb = O.pyramid(A, b), O.pyramid(B, b)
    ref = O.multiply(A, B, b, tau)
    compare_triples(ctx.triples(), ref.triples, pa, pb, d, tau)
    compare_triples(ctx.triples(hi=True), _hi_set(A, B, b, tau_h, ref.triples), pa, pb, d, tau_h)
    if st["tie_band"] == 0 and st["tie_band_hi"] == 0:
        assert st["leaf_triples"] == m
        assert st["hi_products"] == exact
    assert rel_max_err(C, refC) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f16x3", "tf32x3", "bf16x3"])
def test_tier_everything_one_pass(prec):
    """tier_bits = 40 at tau = 1e-9: every kept product runs hi * hi alone
    (every step lean: no low part is loaded), against the oracle's product
    of the rounded operands."""
    p, away = O.HIGH_PART[prec]
    n, b, tau = 700, 32, 1e-9
    A = _matrix("nonsym", n, seed=3)
    B = _matrix("dense", n, seed=4)
    ctx, C = _run(A, B, b, tau, prec, 40)
    refC, m, exact, rounded = O.multiply_tiered(A, B, b, tau, tau * 2.0 ** 40, p, away)
    assert exact == 0 and ctx.stats()["hi_products"] == 0
    assert rel_max_err(C, refC) <= TOL[prec]
    # and it really is the one-pass arithmetic: further from the exact product
    exactC = O.multiply(A, B, b, tau).C
    assert rel_max_err(C, exactC) > 10 * rel_max_err(C, refC)


@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
def test_tier_alpha_beta(prec):
    p, away = O.HIGH_PART[prec]
    n, b, tau = 520, 32, 1e-4
    A = gen.exp_decay_nonsym(n, 0.85, seed=2)
    B = gen.exp_decay_nonsym(n, 0.85, seed=3)
    C0 = gen.uniform_dense(n, seed=4, symmetric=False)
    _, C = _run(A, B, b, tau, prec, p - 1, alpha=0.5, beta=-2.0, C0=C0)
    refC, _, exact, rounded = O.multiply_tiered(A, B, b, tau, tau * 2.0 ** (p - 1), p, away,
                                                alpha=0.5, beta=-2.0, C=C0)
    assert exact > 0 and rounded > 0
    assert rel_max_err(C, refC) <= TOL[prec]


@pytest.mark.parametrize("prec,b,tau,bits", [("f16x3", 64, 1e-2, 10), ("tf32x3", 32, 3e-3, 10),
                                             ("bf16x3", 128, 1e-2, 14)])
def test_tier_with_slice_cull(prec, b, tau, bits):
    """The sub-leaf cull along k with the precision tier: the precision of
    a kept leaf product is chosen by its leaf norms, its slices kept by
    their panel norms, against the oracle's sliced tiered product (at
    tolerances where both tiers are populated)."""
    p, away = O.HIGH_PART[prec]
    n = 900
    A = _matrix("water", n)
    tau_h = tau * 2.0 ** bits
    ctx, C = _run(A, A, b, tau, prec, bits, slice=16)
    refC, m, kept, tested = O.multiply_sliced(A, A, b, 16, tau, tau_h=tau_h, p=p,
                                              ties_away=away)
    st = ctx.stats()
    assert rel_max_err(C, refC) <= TOL[prec]
    if st["tie_band"] == 0:
        assert st["slice_kept"] == kept and st["leaf_triples"] == m
    assert 0 < st["hi_products"] < st["leaf_triples"]


def test_tier_deterministic():
    A = _matrix("water", 1000)
    _, C1 = _run(A, A, 64, 1e-3, "f16x3", 10)
    _, C2 = _run(A, A, 64, 1e-3, "f16x3", 10)
    np.testing.assert_array_equal(C1, C2)


@pytest.mark.parametrize("prec,b,slice", [("f16x3", 64, 0), ("tf32x3", 16, 0),
                                          ("bf16x3", 32, 0), ("f16x3", 64, 16)])
def test_tier_batched_equals_single_and_oracle(prec, b, slice):
    """A mixed batch under the precision tier: every product equals the same
    product run alone bit for bit, and the oracle's tiered product."""
    import paper_1203_1692_gb300 as P
    p, away = O.HIGH_PART[prec]
    bits = p - 1
    rng = np.random.default_rng(7)
    cases = []
    for i, n in enumerate([300, 777, 1024, 129, 1500]):
        lam = float(rng.uniform(0.8, 0.95))
        A = gen.exp_decay(n, lam, seed=100 + i)
        tau = [1e-5, 1e-3, 1e-4][i % 3]
        cases.append((A, tau))
    ctx = P.Context(leaf=b, precision=prec, tier_bits=bits, slice=slice)
    mats = [torch.from_numpy(A).cuda() for A, _ in cases]
    trees = [ctx.build_norms(M) for M in mats]
    Cs = ctx.multiply_batched(trees, trees, [t for _, t in cases])
    torch.cuda.synchronize()
    for q, ((A, tau), C) in enumerate(zip(cases, Cs)):
        _, C1 = _run(A, A, b, tau, prec, bits, slice=slice)
        assert np.array_equal(C.cpu().numpy(), C1)
        if slice:
            refC = O.multiply_sliced(A, A, b, 16, tau, tau_h=tau * 2.0 ** bits, p=p,
                                     ties_away=away)[0]
        else:
            refC = O.multiply_tiered(A, A, b, tau, tau * 2.0 ** bits, p, away)[0]
        assert rel_max_err(C.cpu().numpy(), refC) <= TOL[prec]
        st = ctx.stats_item(q)
        assert 0 <= st["hi_products"] <= st["leaf_triples"]


def test_tier_host_entry_point_equals_device_multiply():
    import paper_1203_1692_gb300 as P
    n, b, tau = 2600, 64, 1e-4
    A = gen.water_like(n // 25, 25, seed=5)
    _, Cd = _run(A, A, b, tau, "f16x3", 10)
    ctx = P.Context(leaf=b, precision="f16x3", tier_bits=10)
    Ch = np.zeros((n, n), dtype=np.float32)
    ctx.multiply_host(A, None, tau, C=Ch)
    assert np.array_equal(Ch, Cd)


def _settled():
    import bench
    return bench.SETTLED["water7500"]


@pytest.mark.slow
@pytest.mark.parametrize("b,tau,bits", [(64, 1e-3, 10), (128, 1e-3, 12), (64, 3e-3, 14),
                                        _settled()])
def test_tier_water_like_n7500(b, tau, bits):
    """The water-like n = 7500 workload at the tolerances and tiers the
    bench searches, including the configuration it settles on and times:
    the whole kept set and the full-split set against the oracle's flat
    enumeration and leaf norms, and sampled C blocks against the oracle's
    tiered blocks."""
    A = gen.water_like()
    n = A.shape[0]
    p, away = O.HIGH_PART["f16x3"]
    tau_h = tau * 2.0 ** bits
    ctx, C = _run(A, A, b, tau, "f16x3", bits)
    st = ctx.stats()
    pa = O.pyramid(A, b)
    d = O.depth(n, b)
    flat = O.cull_linkless(pa, pa, d, tau)
    assert compare_triples_large(ctx.triples(), flat, pa, pa, d, tau) <= st["tie_band"]
    assert compare_triples_large(ctx.triples(hi=True), _hi_set(A, A, b, tau_h, flat), pa, pa,
                                 d, tau_h) <= st["tie_band_hi"]
    assert 0 < st["hi_products"] < st["leaf_triples"]
    ij = sample_blocks(n, b, 24)
    ref, _ = O.blocks(A, A, b, tau, ij, pa, pa, tau_h=tau_h, p=p, ties_away=away)
    got = blocks_from(C, ij, b, n)
    assert float(np.abs(got - ref).max() / np.abs(ref).max()) <= TOL["f16x3"]
