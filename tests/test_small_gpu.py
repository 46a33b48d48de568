"""The fused small-product path: FP32 products of at most 128 leaves per side
run the cull, the grouping and the leaf products in one launch.  A leaf
triple survives the tier-by-tier cull (Eqs. (product), (norm_condition)) iff
its own leaf norms pass the test, since a parent's norm is never below a
child's; so the fused path must give the staged launches' triples, per-tier
counts, tie band and C bit for bit, and the oracle's within the FP32 bar."""
import numpy as np
import pytest

import spamm_inputs as gen
from oracle import oracle as O
from tests.spamm_check import compare_triples, rel_max_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(A, B, b, tau, staged, alpha=1.0, beta=0.0, C0=None):
    import paper_1203_1692_gb300 as P
    ctx = P.Context(leaf=b, precision="fp32", staged=staged)
    ta = ctx.build_norms(torch.from_numpy(A).cuda())
    tb = ta if B is A else ctx.build_norms(torch.from_numpy(B).cuda())
    C = torch.from_numpy(C0.copy()).cuda() if C0 is not None else None
    C = ctx.multiply(ta, tb, tau, alpha, beta, C)
    torch.cuda.synchronize()
    return ctx, C.cpu().numpy()


CASES = [(1024, 16, "exp", 1e-6), (1000, 16, "exp", 1e-4), (2048, 16, "exp", 1e-6),
         (515, 16, "alg", 1e-5), (700, 32, "water", 1e-3), (4096, 32, "exp", 1e-6),
         (129, 16, "exp", 1e-6), (16, 16, "exp", 0.0), (1, 16, "exp", 0.0),
         (300, 64, "dense", 0.0), (333, 16, "dense", 0.0)]


def _matrix(kind, n, seed=0):
    if kind == "exp":
        return gen.exp_decay(n, 0.9, seed=seed)
    if kind == "alg":
        return gen.algebraic_decay(n, seed=seed)
    if kind == "water":
        return gen.water_like(n // 25, 25, seed=seed)
    return gen.uniform_dense(n, seed=seed, symmetric=False)


@pytest.mark.parametrize("n,b,kind,tau", CASES)
def test_fused_equals_staged_and_oracle(n, b, kind, tau):
    A = _matrix(kind, n)
    B = _matrix("exp", n, seed=1) if kind == "dense" else A
    fused, Cf = _run(A, B, b, tau, staged=False)
    staged, Cs = _run(A, B, b, tau, staged=True)
    sf, ss = fused.stats(), staged.stats()
    assert np.array_equal(Cf, Cs)
    for key in ("tier_candidates", "tier_kept", "leaf_triples", "tie_band", "active_steps",
                "kept_flops", "kept_flops_clipped"):
        assert sf[key] == ss[key], key
    tf = fused.triples()
    assert sorted(map(tuple, tf.tolist())) == sorted(map(tuple, staged.triples().tolist()))
    if n * n <= 1100 ** 2:
        ref = O.multiply(A, B, b, tau)
        compare_triples(tf, ref.triples, O.pyramid(A, b), O.pyramid(B, b), O.depth(n, b), tau)
        assert rel_max_err(Cf, ref.C) <= 1e-5
        if sf["tie_band"] == 0:
            assert sf["tier_kept"] == ref.kept.tolist()
            assert sf["tier_candidates"] == ref.cand.tolist()


def test_fused_alpha_beta_and_nonfinite():
    n, b, tau = 600, 16, 1e-5
    A = gen.exp_decay_nonsym(n, 0.85, seed=2)
    B = gen.exp_decay_nonsym(n, 0.85, seed=3)
    C0 = gen.uniform_dense(n, seed=4, symmetric=False)
    _, Cf = _run(A, B, b, tau, False, alpha=0.5, beta=-2.0, C0=C0)
    _, Cs = _run(A, B, b, tau, True, alpha=0.5, beta=-2.0, C0=C0)
    assert np.array_equal(Cf, Cs)
    ref = O.multiply(A, B, b, tau, alpha=0.5, beta=-2.0, C=C0)
    assert rel_max_err(Cf, ref.C) <= 1e-5
    # a NaN: NONFINITE, C untouched
    import paper_1203_1692_gb300 as P
    A[5, 7] = np.nan
    ctx = P.Context(leaf=b, precision="fp32")
    t = ctx.build_norms(torch.from_numpy(A).cuda())
    C = torch.from_numpy(C0.copy()).cuda()
    with pytest.raises(P.SpammError) as err:
        ctx.multiply(t, t, tau, 1.0, 0.0, C)
    assert err.value.status == P._abi.SPAMM_ERR_NONFINITE
    assert np.array_equal(C.cpu().numpy(), C0)


def test_fused_path_in_a_cuda_graph():
    """The whole small step (norm tree + fused multiply) captured once and
    replayed gives the eager result."""
    import paper_1203_1692_gb300 as P
    n, b, tau = 1024, 16, 1e-6
    A = torch.from_numpy(gen.exp_decay(n, 0.9, seed=0)).cuda()
    ctx = P.Context(leaf=b, precision="fp32", checked=True)
    tree = ctx.build_norms(A)
    C = torch.empty_like(A)
    ctx.multiply(tree, tree, tau, C=C)
    ref = C.clone()
    ctx.set_checked(False)
    s = torch.cuda.Stream()
    P._abi.spamm_set_stream(ctx.handle, s.cuda_stream)
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        tree.rebuild(A)
        ctx.multiply(tree, tree, tau, C=C)
    C.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(C, ref)
