"""Batched products through spamm_multiply_batched (C ABI).

A batch of independent products of different n (the leaf products of all of
them in one persistent launch on the tensor-core precisions) must give, for
every product, the same C bit for bit as a single spamm_multiply of it, and
the oracle's C within the precision's tolerance (Sec. III.D: each product is
its own recursion; the batch only shares the launch)."""
import numpy as np
import pytest

import spamm_inputs as gen
from oracle import oracle
from tests.spamm_check import rel_max_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "tf32x3": 1e-5, "f16x3": 1e-5, "bf16x3": 1e-4, "tf32": 5e-3}


def _mix(seed=0):
    """Products of mixed size, decay and threshold (ragged tails included)."""
    rng = np.random.default_rng(seed)
    out = []
    for i, n in enumerate([300, 512, 777, 1024, 129, 1500]):
        lam = float(rng.uniform(0.8, 0.95))
        A = gen.exp_decay(n, lam, seed=100 + i)
        B = gen.exp_decay_nonsym(n, lam, seed=200 + i) if i % 2 else A
        tau = [1e-7, 1e-5, 1e-3][i % 3]
        alpha, beta = [(1.0, 0.0), (-0.5, 2.0), (2.0, 1.0)][i % 3]
        C0 = gen.uniform_dense(n, seed=300 + i, symmetric=False)
        out.append((A, B, tau, alpha, beta, C0))
    return out


def _single(P, prec, case):
    A, B, tau, alpha, beta, C0 = case
    ctx = P.Context(leaf=16, precision=prec)
    ta = ctx.build_norms(torch.from_numpy(A).cuda())
    tb = ctx.build_norms(torch.from_numpy(B).cuda())
    C = torch.from_numpy(C0.copy()).cuda()
    ctx.multiply(ta, tb, tau, alpha, beta, C)
    torch.cuda.synchronize()
    return C.cpu().numpy(), ctx.stats()["leaf_triples"]


def _batched(P, prec, cases, ctx=None, leaf=16, slice=0):
    ctx = ctx or P.Context(leaf=leaf, precision=prec, slice=slice)
    keep = []
    As, Bs, Cs = [], [], []
    for A, B, tau, alpha, beta, C0 in cases:
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        keep += [dA, dB]
        As.append(ctx.build_norms(dA))
        Bs.append(ctx.build_norms(dB))
        Cs.append(torch.from_numpy(C0.copy()).cuda())
    ctx.multiply_batched(As, Bs, [c[2] for c in cases], [c[3] for c in cases],
                         [c[4] for c in cases], Cs)
    torch.cuda.synchronize()
    return [C.cpu().numpy() for C in Cs], ctx


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "fp32", "tf32", "f16x3"])
def test_batched_equals_single_bit_for_bit(prec):
    import paper_1203_1692_gb300 as P
    cases = _mix()
    got, ctx = _batched(P, prec, cases)
    total = 0
    for case, C in zip(cases, got):
        ref, m = _single(P, prec, case)
        total += m
        assert np.array_equal(C, ref)
    assert ctx.stats()["leaf_triples"] == total


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "f16x3"])
def test_batched_matches_oracle(prec):
    import paper_1203_1692_gb300 as P
    cases = _mix(seed=1)[:4]
    got, _ = _batched(P, prec, cases)
    for (A, B, tau, alpha, beta, C0), C in zip(cases, got):
        ref = oracle.multiply(A, B, 16, tau, alpha=alpha, beta=beta, C=C0)
        assert rel_max_err(C, ref.C) <= TOL[prec]


@pytest.mark.parametrize("prec,leaf", [("f16x3", 64), ("f16x3", 128), ("tf32x3", 64),
                                       ("bf16x3", 128)])
def test_batched_slice_cull_matches_oracle(prec, leaf):
    """The configuration the batch-of-64 workload runs (leaf 64 or 128, the
    sub-leaf cull along k in slices of 16): every product of a mixed batch
    against the oracle's sliced product (reading R14 of the SpAMM(4x4)
    cull), with its kept slice count."""
    import paper_1203_1692_gb300 as P
    cases = _mix(seed=4)
    got, ctx = _batched(P, prec, cases, leaf=leaf, slice=16)
    for p, ((A, B, tau, alpha, beta, C0), C) in enumerate(zip(cases, got)):
        refC, m, kept, _ = oracle.multiply_sliced(A, B, leaf, 16, tau, alpha=alpha, beta=beta,
                                                  C=C0)
        assert rel_max_err(C, refC) <= TOL[prec]
        st = ctx.stats_item(p)
        if st["tie_band"] == 0:
            assert st["leaf_triples"] == m
            assert st["slice_kept"] == kept


def test_batched_more_than_one_launch_and_reuse():
    """70 products (above the 64 of one launch), then the same context again
    with other inputs: sub-contexts are reused and nothing carries over."""
    import paper_1203_1692_gb300 as P
    rng = np.random.default_rng(5)
    ctx = P.Context(leaf=16, precision="tf32x3")
    for rep in range(2):
        cases = []
        for i in range(70):
            n = int(rng.integers(64, 400))
            A = gen.exp_decay(n, 0.85, seed=1000 * rep + i)
            cases.append((A, A, 1e-5, 1.0, 0.0, np.zeros((n, n), np.float32)))
        got, _ = _batched(P, "tf32x3", cases, ctx=ctx)
        for case, C in zip(cases[::9], got[::9]):
            ref, _ = _single(P, "tf32x3", case)
            assert np.array_equal(C, ref)


def test_batched_pool_growth_in_checked_mode():
    """Sub-context pools start at the configured (tiny) size and grow."""
    import paper_1203_1692_gb300 as P
    cases = _mix(seed=2)[:3]
    ctx = P.Context(leaf=16, precision="tf32x3", pool_bytes=16384)
    got, ctx = _batched(P, "tf32x3", cases, ctx=ctx)
    st = ctx.stats()
    assert st["status"] == 0
    assert st["pool_bytes"] >= st["pool_needed_bytes"]
    for case, C in zip(cases, got):
        ref, _ = _single(P, "tf32x3", case)
        assert np.array_equal(C, ref)


def test_batched_deterministic_and_graph_capturable():
    import paper_1203_1692_gb300 as P
    cases = _mix(seed=3)
    ctx = P.Context(leaf=16, precision="bf16x3")
    first, _ = _batched(P, "bf16x3", cases, ctx=ctx)
    # replay the same batch in a CUDA graph (unchecked mode, sub-contexts exist)
    As, Bs, Cs, keep = [], [], [], []
    for A, B, tau, alpha, beta, C0 in cases:
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        keep += [dA, dB]
        As.append(ctx.build_norms(dA))
        Bs.append(ctx.build_norms(dB))
        Cs.append(torch.from_numpy(C0.copy()).cuda())
    C0s = [C.clone() for C in Cs]
    ctx.set_checked(False)
    s = torch.cuda.Stream()
    P._abi.spamm_set_stream(ctx.handle, s.cuda_stream)
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        ctx.multiply_batched(As, Bs, [c[2] for c in cases], [c[3] for c in cases],
                             [c[4] for c in cases], Cs)
    for _ in range(2):
        for C, C0 in zip(Cs, C0s):
            C.copy_(C0)
        g.replay()
        torch.cuda.synchronize()
        for C, ref in zip(Cs, first):
            assert np.array_equal(C.cpu().numpy(), ref)


def test_batched_rejects_bad_arguments():
    import paper_1203_1692_gb300 as P
    ctx = P.Context(leaf=16, precision="tf32x3")
    other = P.Context(leaf=32, precision="tf32x3")
    A = torch.from_numpy(gen.exp_decay(256, 0.9, seed=1)).cuda()
    ta, tb = ctx.build_norms(A), other.build_norms(A)
    with pytest.raises(P.SpammError):
        ctx.multiply_batched([ta], [tb], [1e-6])
    with pytest.raises(P.SpammError):
        ctx.multiply_batched([ta], [ta], [-1.0])
    ctx.multiply_batched([], [], [])    # empty batch: nothing to do


def test_rebuild_batched_matches_single_builds():
    """spamm_tree_rebuild_batched gives every tree the norms a fresh
    spamm_build_norms gives (Sec. II.A), bit for bit."""
    import paper_1203_1692_gb300 as P
    ctx = P.Context(leaf=32, precision="bf16x3")
    mats = [torch.from_numpy(gen.exp_decay(n, 0.88, seed=40 + n)).cuda()
            for n in (100, 640, 1000, 1333, 64, 2048, 700, 900, 515)]
    trees = [ctx.build_norms(torch.zeros_like(A)) for A in mats]
    ctx.rebuild_batched(trees, mats)
    for t, A in zip(trees, mats):
        assert np.array_equal(t.norms(), ctx.build_norms(A).norms())


def test_decay_estimate_on_the_device_matches_the_oracle_pyramid():
    """The autotuner's decay estimate reads the library's own norm pyramid;
    it equals the same share computed from the oracle's pyramid."""
    from paper_1203_1692_gb300 import autotune
    for n, lam in ((700, 0.8), (2048, 0.95)):
        A = gen.exp_decay(n, lam, seed=3)
        ref = autotune.decay_from_pyramid(oracle.pyramid(A, 64), oracle.depth(n, 64))
        got = autotune.decay_estimate(torch.from_numpy(A).cuda())
        assert abs(got - ref) <= 1e-9 * ref
