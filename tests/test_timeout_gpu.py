"""Failure detection on the device without a fault: the tensor-core leaf
kernel bounds every wait of its pipeline, and a wait that runs out makes it
give up cleanly (TIMEOUT status, its copies and MMAs drained, tensor memory
freed, the context still usable).  The test shortens the bound to 1 ns, so
the first wait that is not satisfied at once runs out; nothing here faults
or hangs the GPU."""
import pytest

import spamm_inputs as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,b,bits", [("f16x3", 64, 0), ("f16x3", 128, 16), ("tf32x3", 32, 0)])
def test_short_wait_bound_gives_timeout_and_the_context_recovers(prec, b, bits):
    import paper_1203_1692_gb300 as P
    A = torch.from_numpy(gen.water_like(120, 25, seed=3)).cuda()     # n = 3000
    ref_ctx = P.Context(leaf=b, precision=prec, tier_bits=bits)
    rt = ref_ctx.build_norms(A)
    ref = ref_ctx.multiply(rt, rt, 1e-4)
    torch.cuda.synchronize()

    ctx = P.Context(leaf=b, precision=prec, tier_bits=bits)
    tree = ctx.build_norms(A)
    ctx.set_wait_limit(1)
    with pytest.raises(P.SpammError) as err:
        ctx.multiply(tree, tree, 1e-4)
    assert err.value.status == P._abi.SPAMM_ERR_TIMEOUT
    assert ctx.stats(raise_on_error=False)["status"] == P._abi.SPAMM_ERR_TIMEOUT
    # the default bound again: the same context gives the reference result
    ctx.set_wait_limit(0)
    C = ctx.multiply(tree, tree, 1e-4)
    torch.cuda.synchronize()
    assert ctx.stats()["status"] == 0
    assert torch.equal(C, ref)
    # and the device is healthy for other work
    x = torch.ones(1024, device="cuda")
    assert float(x.sum()) == 1024.0
