"""Sparsified storage (Sec. II.D, drop tolerance) through spamm_sparsify:
leaves whose product with the largest operand norm fails the SpAMM test are
dropped, the rest stored band by band, and the tensor-core packs hold only
pieces inside the bands."""
import numpy as np
import pytest

import spamm_inputs as gen
from oracle import oracle as O
from tests.spamm_check import as_set, rel_max_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"tf32x3": 1e-5, "f16x3": 1e-5, "bf16x3": 1e-4}


def _n2(A):
    return float((A.astype(np.float64) ** 2).sum())


@pytest.mark.parametrize("prec,b", [("tf32x3", 16), ("tf32x3", 64), ("bf16x3", 32),
                                    ("tf32x3", 128), ("f16x3", 64)])
@pytest.mark.parametrize("n,tau", [(1000, 1e-6), (777, 1e-4), (1500, 1e-8)])
def test_sparsified_product_equals_dense_product(prec, b, n, tau):
    """At the consistent tolerance the sparsified operands keep exactly the
    leaf products of the dense ones, so C is the same bit for bit."""
    import paper_1203_1692_gb300 as P
    A = gen.exp_decay(n, 0.85, seed=n)
    B = gen.exp_decay_nonsym(n, 0.9, seed=n + 1)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    ctx = P.Context(leaf=b, precision=prec)
    C_dense = ctx.multiply(ctx.build_norms(dA), ctx.build_norms(dB), tau)
    ta = ctx.sparsify(dA, tau, _n2(B))
    tb = ctx.sparsify(dB, tau, _n2(A))
    C = ctx.multiply(ta, tb, tau)
    torch.cuda.synchronize()
    assert torch.equal(C, C_dense)
    nl = -(-n // b)
    assert 0 < ta.stored_leaves < nl * nl
    assert ta.bytes < ctx.build_norms(dA).bytes


def test_sparsified_against_the_oracle_at_a_coarser_drop():
    """Dropping more than the consistent tolerance (partner norm scaled up)
    changes the product; the GPU then matches the oracle's product of the
    oracle's sparsified operands."""
    import paper_1203_1692_gb300 as P
    n, b, tau = 900, 32, 1e-5
    A = gen.exp_decay(n, 0.8, seed=3)
    big = 1e6 * _n2(A)
    As, m = O.sparsify(A, b, tau, big)
    dA = torch.from_numpy(A).cuda()
    ctx = P.Context(leaf=b, precision="tf32x3")
    t = ctx.sparsify(dA, tau, big)
    assert t.stored_leaves == m
    C = ctx.multiply(t, t, tau)
    ref = O.multiply(As, As, b, tau)
    assert rel_max_err(C.cpu().numpy(), ref.C) <= TOL["tf32x3"]
    assert as_set(ctx.triples()) == as_set(ref.triples)


def test_mixed_sparse_and_dense_operands_and_batches():
    import paper_1203_1692_gb300 as P
    n, tau = 1024, 1e-6
    A = gen.exp_decay(n, 0.9, seed=5)
    dA = torch.from_numpy(A).cuda()
    ctx = P.Context(leaf=64, precision="tf32x3")
    dense = ctx.build_norms(dA)
    sp = ctx.sparsify(dA, tau, 0.0)
    ref = ctx.multiply(dense, dense, tau)
    assert torch.equal(ctx.multiply(sp, dense, tau), ref)
    assert torch.equal(ctx.multiply(dense, sp, tau), ref)
    Cs = ctx.multiply_batched([sp, dense, sp], [sp, sp, dense], [tau] * 3)
    for C in Cs:
        assert torch.equal(C, ref)


def test_sparsified_storage_is_linear_in_n():
    """For a banded decay the sparsified tree's bytes grow ~linearly with n
    (the dense tree's quadratically)."""
    import paper_1203_1692_gb300 as P
    ctx = P.Context(leaf=32, precision="tf32x3")
    sizes = {}
    for n in (2048, 4096):
        dA = torch.from_numpy(gen.exp_decay(n, 0.8, seed=1)).cuda()
        sizes[n] = (ctx.sparsify(dA, 1e-6, 0.0).bytes, ctx.build_norms(dA).bytes)
    sp_ratio = sizes[4096][0] / sizes[2048][0]
    dn_ratio = sizes[4096][1] / sizes[2048][1]
    assert sp_ratio < 2.6 and dn_ratio > 3.5


def test_sparsify_rejects_rebuild_and_fp32():
    import paper_1203_1692_gb300 as P
    dA = torch.from_numpy(gen.exp_decay(300, 0.9, seed=2)).cuda()
    ctx = P.Context(leaf=16, precision="tf32x3")
    t = ctx.sparsify(dA, 1e-6, 0.0)
    with pytest.raises(P.SpammError):
        t.rebuild(dA)
    with pytest.raises(P.SpammError):
        P.Context(leaf=16, precision="fp32").sparsify(dA, 1e-6, 0.0)


@pytest.mark.parametrize("prec,b", [("tf32x3", 32), ("f16x3", 64), ("bf16x3", 16)])
def test_resparsify_in_place_equals_a_fresh_tree(prec, b):
    """spamm_sparsify_into gives the fresh tree's product bit for bit, when
    the new bands fit (narrower decay: the storage is reused) and when they
    do not (wider decay: it grows), and keeps its storage on a second call
    with the same matrix."""
    import paper_1203_1692_gb300 as P
    n, tau = 1200, 1e-6
    ctx = P.Context(leaf=b, precision=prec)
    mats = [gen.exp_decay(n, lam, seed=s) for lam, s in ((0.85, 1), (0.7, 2), (0.93, 3))]
    t = None
    for A in mats:
        dA = torch.from_numpy(A).cuda()
        fresh = ctx.sparsify(dA, tau, 0.0)
        C_ref = ctx.multiply(fresh, fresh, tau)
        if t is None:
            t = ctx.sparsify(dA, tau, 0.0)
        else:
            before = t.bytes
            t.resparsify(dA, tau, 0.0)
            # reused when the bands fit, grown beyond the need when not
            assert t.bytes == before or t.bytes > fresh.bytes
        assert t.stored_leaves == fresh.stored_leaves
        C = ctx.multiply(t, t, tau)
        torch.cuda.synchronize()
        assert torch.equal(C, C_ref)
        kept = t.bytes
        t.resparsify(dA, tau, 0.0)
        assert t.bytes == kept
        assert torch.equal(ctx.multiply(t, t, tau), C_ref)
        fresh.close()


def test_resparsify_against_the_oracle_and_errors():
    """A re-sparsified tree matches the oracle's sparsified product; a NaN
    leaves the tree reporting NONFINITE until a good matrix is sparsified
    into it; a dense tree, another n or another context is refused."""
    import paper_1203_1692_gb300 as P
    n, b, tau = 900, 32, 1e-5
    A = gen.exp_decay(n, 0.8, seed=3)
    big = 1e6 * _n2(A)
    dA = torch.from_numpy(A).cuda()
    ctx = P.Context(leaf=b, precision="tf32x3")
    t = ctx.sparsify(torch.from_numpy(gen.exp_decay(n, 0.9, seed=4)).cuda(), tau, 0.0)
    t.resparsify(dA, tau, big)
    As, m = O.sparsify(A, b, tau, big)
    assert t.stored_leaves == m
    C = ctx.multiply(t, t, tau)
    ref = O.multiply(As, As, b, tau)
    assert rel_max_err(C.cpu().numpy(), ref.C) <= TOL["tf32x3"]
    bad = A.copy()
    bad[10, 20] = np.nan
    with pytest.raises(P.SpammError) as err:
        t.resparsify(torch.from_numpy(bad).cuda(), tau, 0.0)
    assert err.value.status == P._abi.SPAMM_ERR_NONFINITE
    with pytest.raises(P.SpammError) as err:
        ctx.multiply(t, t, tau)
    assert err.value.status == P._abi.SPAMM_ERR_NONFINITE
    t.resparsify(dA, tau, big)
    assert torch.equal(ctx.multiply(t, t, tau), C)
    with pytest.raises(ValueError):
        t.resparsify(torch.zeros(n + 1, n + 1, device="cuda"), tau, 0.0)
    with pytest.raises(P.SpammError):
        P._abi.spamm_sparsify_into(ctx.handle, ctx.build_norms(dA).handle, dA.data_ptr(), n,
                                   tau, 0.0)
    other = P.Context(leaf=b, precision="tf32x3")
    with pytest.raises(P.SpammError):
        P._abi.spamm_sparsify_into(other.handle, t.handle, dA.data_ptr(), n, tau, 0.0)
