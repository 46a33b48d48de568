"""The allocation-free entry point, spamm_multiply_static, called through the
C ABI.

It exists for callers that cannot allocate device memory (a host framework
or plugin that owns all device memory through its own allocator or memory
cap, or a loop that must not pay cudaMalloc's implicit synchronisation); all
of its scratch lives in a static device array.  Its output must agree with
the regular entry points (spamm_build_norms + spamm_multiply, FP32 leaf
products) within the FP32 parity tolerance, on two calls in a row with
different inputs, so that nothing from the first call leaks into the second.
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import spamm_inputs as gen
from oracle import oracle as O
from tests.spamm_check import blocks_from, sample_blocks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5   # max|dC| / max|C|, the FP32 parity bar


def _regular(A, B, tau, alpha, beta, C0):
    import paper_1203_1692_gb300 as P
    ctx = P.Context(leaf=16, precision="fp32")
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    ta, tb = ctx.build_norms(dA), ctx.build_norms(dB)
    C = torch.from_numpy(C0.copy()).cuda()
    ctx.multiply(ta, tb, tau, alpha, beta, C)
    torch.cuda.synchronize()
    return C.cpu().numpy()


def _static(A, B, tau, alpha, beta, C0):
    from paper_1203_1692_gb300 import _abi
    n = A.shape[0]
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    C = torch.from_numpy(C0.copy()).cuda()
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    _abi.spamm_multiply_static(dA.data_ptr(), n, dB.data_ptr(), n, n, tau, alpha, beta,
                               C.data_ptr(), n, stream, status.data_ptr())
    torch.cuda.synchronize()
    return C.cpu().numpy(), int(status.item())


def _rel(C, ref):
    ref = ref.astype(np.float64)
    return float(np.abs(C.astype(np.float64) - ref).max() / np.abs(ref).max())


def test_static_matches_regular_entry_point_twice_in_a_row():
    cases = [
        (gen.exp_decay(1000, 0.9, seed=1), gen.exp_decay(1000, 0.9, seed=1), 1e-4, 1.0, 0.0),
        (gen.exp_decay_nonsym(700, 0.85, seed=2), gen.uniform_dense(700, seed=3, symmetric=False),
         1e-6, -0.5, 2.0),
    ]
    for A, B, tau, alpha, beta in cases:
        n = A.shape[0]
        C0 = gen.uniform_dense(n, seed=7, symmetric=False)
        ref = _regular(A, B, tau, alpha, beta, C0)
        got, status = _static(A, B, tau, alpha, beta, C0)
        assert status == 0
        assert _rel(got, ref) <= TOL


def test_static_allocates_no_device_memory_after_setup():
    n = 512
    A = gen.exp_decay(n, 0.9, seed=4)
    C0 = np.zeros((n, n), dtype=np.float32)
    _static(A, A, 1e-6, 1.0, 0.0, C0)          # first call on the device: set-up
    from paper_1203_1692_gb300 import _abi
    dA = torch.from_numpy(A).cuda()
    C = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        _abi.spamm_multiply_static(dA.data_ptr(), n, dA.data_ptr(), n, n, 1e-6, 1.0, 0.0,
                                   C.data_ptr(), n, stream, 0)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    ref = _regular(A, A, 1e-6, 1.0, 0.0, C0)
    assert _rel(C.cpu().numpy(), ref) <= TOL


def test_static_accepts_its_maximum_and_rejects_beyond():
    from paper_1203_1692_gb300 import _abi
    L = _abi.lib()
    n = 4096                                   # the stated maximum
    Z = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    C = torch.ones((n, n), dtype=torch.float32, device="cuda")
    st = L.spamm_multiply_static(ctypes.c_void_p(Z.data_ptr()), n, ctypes.c_void_p(Z.data_ptr()),
                                 n, n, 1e-6, 1.0, 0.5, ctypes.c_void_p(C.data_ptr()), n,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), None)
    torch.cuda.synchronize()
    assert st == _abi.SPAMM_OK
    assert float(C.max()) == 0.5 and float(C.min()) == 0.5   # A = 0: C = beta * C
    x = torch.zeros((1,), dtype=torch.float32, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    n = 4097
    st = L.spamm_multiply_static(p, n, p, n, n, 1e-6, 1.0, 0.0, p, n, None, None)
    assert st == _abi.SPAMM_ERR_UNSUPPORTED
    st = L.spamm_multiply_static(p, 4, p, 4, 8, 1e-6, 1.0, 0.0, p, 8, None, None)
    assert st == _abi.SPAMM_ERR_INVALID_ARG


def test_static_matches_oracle():
    """The allocation-free product against the FP64 oracle directly (Eqs.
    (product), (norm_condition), Algorithm 1), with alpha and beta."""
    n, tau, alpha, beta = 900, 1e-5, 0.75, -1.5
    A = gen.exp_decay_nonsym(n, 0.85, seed=11)
    B = gen.exp_decay(n, 0.9, seed=12)
    C0 = gen.uniform_dense(n, seed=13, symmetric=False)
    ref = O.multiply(A, B, 16, tau, alpha=alpha, beta=beta, C=C0)
    got, status = _static(A, B, tau, alpha, beta, C0)
    assert status == 0
    assert _rel(got, ref.C) <= TOL


def test_static_worst_case_at_its_maximum():
    """n = 4096 at tau = 0 on a dense matrix: every block product is kept,
    which is the case the static scratch is sized for (full frontiers at
    every tier, every tile with all its steps).  Sampled C blocks against
    the oracle, the whole C against the regular entry point, and the
    regular entry point's kept count against the oracle's (all (n/16)^3)."""
    import paper_1203_1692_gb300 as P
    n, b, tau = 4096, 16, 0.0
    A = gen.uniform_dense(n, seed=21, symmetric=False)
    B = gen.uniform_dense(n, seed=22, symmetric=False)
    C0 = np.zeros((n, n), dtype=np.float32)
    got, status = _static(A, B, tau, 1.0, 0.0, C0)
    assert status == 0
    ij = sample_blocks(n, b, 24)
    ref, kept = O.blocks(A, B, b, tau, ij)
    assert kept == len(ij) * (n // b)
    blk = blocks_from(got, ij, b, n)
    assert float(np.abs(blk - ref).max() / np.abs(ref).max()) <= TOL
    ctx = P.Context(leaf=b, precision="fp32")
    ta = ctx.build_norms(torch.from_numpy(A).cuda())
    tb = ctx.build_norms(torch.from_numpy(B).cuda())
    C = ctx.multiply(ta, tb, tau)
    torch.cuda.synchronize()
    assert ctx.stats()["leaf_triples"] == (n // b) ** 3
    assert _rel(got, C.cpu().numpy()) <= TOL


def test_static_non_finite_input_reports_status_and_leaves_C():
    """A NaN in A: the device status word reads 2 (non-finite input) and C
    is left as it was."""
    n = 300
    A = gen.exp_decay(n, 0.9, seed=31)
    A[17, 123] = np.nan
    C0 = gen.uniform_dense(n, seed=32, symmetric=False)
    got, status = _static(A, A, 1e-6, 1.0, 0.5, C0)
    assert status == 2
    assert np.array_equal(got, C0)
