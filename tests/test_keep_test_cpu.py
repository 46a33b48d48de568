"""The cull's keep test decides most pairs from the FP64 exponent fields
alone and multiplies only near the threshold.  Emulated here with the same
integer arithmetic on the bit patterns and checked against the plain
comparison fl(a*b) >= tau^2 for squared leaf norms (sums of squares of FP32
values: normal doubles in [2^-298, 2^278]), including products within a few
ulps of the threshold and of the tie band's edges."""
import struct

import numpy as np
import pytest


def _bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _thresh(tau, rel=1e-6):
    tau2 = tau * tau
    lo2 = tau2 * (1.0 - rel) * (1.0 - rel)
    hi2 = tau2 * (1.0 + rel) * (1.0 + rel)
    return tau2, lo2, hi2, _bits(lo2) >> 52, _bits(hi2) >> 52


def _keep(a, b, th):
    tau2, lo2, hi2, e_lo, e_hi = th
    ua, ub = _bits(a), _bits(b)
    if ua == 0 or ub == 0:
        return False
    s = (ua >> 52) + (ub >> 52) - 1023
    if s >= 1 and s >= e_hi + 1:
        return True
    if s + 2 < e_lo:
        return False
    return a * b >= tau2


def _plain(a, b, tau2):
    return a > 0 and b > 0 and a * b >= tau2


@pytest.mark.parametrize("tau", [1e-10, 1e-6, 1e-4, 0.37, 1.0, 1e3])
def test_exponent_shortcut_equals_plain_comparison(tau):
    th = _thresh(tau)
    rng = np.random.default_rng(int(tau * 1e6) % 1000)
    # random norms over the whole range squared FP32 leaf norms can take
    e = rng.uniform(-298, 278, size=(20000, 2))
    ab = np.exp2(e) * rng.uniform(1, 2, size=e.shape)
    for a, b in ab:
        assert _keep(a, b, th) == _plain(a, b, th[0])
    # pairs whose product lands within a few ulps of tau^2 and of the band edges
    for target in (th[0], th[1], th[2]):
        for _ in range(2000):
            a = float(np.exp2(rng.uniform(-100, 100)))
            b = target / a
            for db in (np.nextafter(b, 0), b, np.nextafter(b, np.inf)):
                assert _keep(a, float(db), th) == _plain(a, float(db), th[0])


def test_zero_norms_never_kept():
    th = _thresh(0.0)
    assert not _keep(0.0, 1.0, th) and not _keep(1.0, 0.0, th)
    assert _keep(1e-200, 1e-90, th)          # tau = 0 keeps every non-NULL pair
