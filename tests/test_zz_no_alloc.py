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
