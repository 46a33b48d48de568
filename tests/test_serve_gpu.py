"""Serving chains of squarings X <- X^2 (the paper's test operation, Sec.
IV) through the continuous-batching server: each request's result is the
same, bit for bit, when it runs alone and when it runs in a mix of requests
of other sizes and thresholds that join and leave mid-chain."""
import numpy as np
import pytest

import spamm_inputs as gen
from oracle import oracle as O
from tests.spamm_check import rel_max_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _x0(n, seed):
    A = torch.from_numpy(gen.exp_decay(n, 0.9, seed=seed)).cuda()
    return A / A.abs().sum(1).max()          # spectral radius <= 1


def _requests():
    from paper_1203_1692_gb300.serve import Request
    spec = [(700, 1e-6, 0.0), (1200, 1e-8, 0.0), (300, 1e-6, 0.001), (2000, 1e-8, 0.002),
            (515, 1e-6, 0.05), (900, 1e-8, 0.05)]
    return [Request(rid=i, n=n, tau=tau, squarings=4, arrival=t, X0=_x0(n, 10 + i))
            for i, (n, tau, t) in enumerate(spec)]


@pytest.mark.parametrize("prec,b,bits,asynchronous", [("tf32x3", 16, 0, True),
                                                      ("bf16x3", 32, 0, False),
                                                      ("fp32", 16, 0, True),
                                                      ("f16x3", 64, 10, True)])
def test_result_is_the_same_alone_and_in_the_mix(prec, b, bits, asynchronous):
    """Asynchronous batches (admission while a batch runs) and synchronous
    ones, with and without precision chosen by norm."""
    from paper_1203_1692_gb300.serve import GpuChainExecutor, Server

    def ex():
        return GpuChainExecutor(leaf=b, precision=prec, tier_bits=bits, asynchronous=asynchronous)
    mixed = Server(ex(), budget_bytes=8 << 30)
    done = {r.rid: r for r in mixed.run(_requests())}
    assert max(mixed.batch_sizes) >= 3
    for req in _requests():
        alone = Server(ex(), budget_bytes=8 << 30)
        got = alone.run([req])[0]
        assert torch.equal(got.result, done[req.rid].result)


def test_async_batch_with_overflowing_pools_is_rerun():
    """Sub-context pools that start tiny overflow in the unchecked batch; the
    executor reruns the batch checked and the chain matches a checked run."""
    from paper_1203_1692_gb300.serve import GpuChainExecutor, Server
    ex = GpuChainExecutor(leaf=16, precision="tf32x3")
    ex.ctx.close()
    import paper_1203_1692_gb300 as P
    ex.ctx = P.Context(leaf=16, precision="tf32x3", checked=False, pool_bytes=16384)
    got = {r.rid: r for r in Server(ex, budget_bytes=8 << 30).run(_requests())}
    assert ex.reruns >= 1
    ref = {r.rid: r for r in Server(GpuChainExecutor(leaf=16, precision="tf32x3",
                                                     asynchronous=False),
                                    budget_bytes=8 << 30).run(_requests())}
    for rid in ref:
        assert torch.equal(got[rid].result, ref[rid].result)


def test_one_squaring_matches_the_oracle():
    from paper_1203_1692_gb300.serve import GpuChainExecutor, Request, Server
    X0 = _x0(640, 3)
    srv = Server(GpuChainExecutor(leaf=16, precision="tf32x3"), budget_bytes=1 << 30)
    r = srv.run([Request(rid=0, n=640, tau=1e-6, squarings=1, X0=X0)])[0]
    Xh = X0.cpu().numpy()
    ref = O.multiply(Xh, Xh, 16, 1e-6)
    assert rel_max_err(r.result.cpu().numpy(), ref.C) <= 1e-5
