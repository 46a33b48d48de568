"""The seeded input generators: the device forms of the exponential- and
algebraic-decay generators give the host forms' matrices bit for bit."""
import numpy as np
import pytest

import spamm_inputs as gen
from spamm_inputs import device as D

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("n,lam,seed", [(1, 0.9, 0), (300, 0.85, 3), (777, 0.93, 12345),
                                        (2000, 0.8, 7)])
def test_device_exp_decay_equals_host_on_cpu(n, lam, seed):
    a = gen.exp_decay(n, lam, seed=seed)
    b = D.exp_decay(n, lam, seed=seed, device="cpu").numpy()
    assert np.array_equal(a, b)


def test_exp_decay_is_symmetric_and_decays():
    a = gen.exp_decay(200, 0.8, seed=1)
    assert np.array_equal(a, a.T)
    i, j = np.indices(a.shape)
    assert np.all(np.abs(a) <= 0.8 ** np.abs(i - j) * (1 + 1e-6))


def test_batched_products_ranges():
    ps = gen.batched_products(64, 512, 8192, 0.8, 0.95, seed=0)
    assert len(ps) == 64
    assert all(512 <= n <= 8192 and 0.8 <= lam <= 0.95 for n, lam, _ in ps)
    assert len({s for _, _, s in ps}) == 64


@pytest.mark.gpu
def test_device_exp_decay_equals_host_on_gpu():
    for n, lam, seed in [(1000, 0.9, 1), (4097, 0.82, 5)]:
        a = gen.exp_decay(n, lam, seed=seed)
        b = D.exp_decay(n, lam, seed=seed, device="cuda").cpu().numpy()
        assert np.array_equal(a, b)


@pytest.mark.parametrize("n,seed", [(1, 0), (300, 3), (1025, 12345)])
def test_device_algebraic_decay_equals_host_on_cpu(n, seed):
    a = gen.algebraic_decay(n, seed=seed)
    b = D.algebraic_decay(n, seed=seed, device="cpu").numpy()
    assert np.array_equal(a, b)


@pytest.mark.gpu
def test_device_algebraic_decay_equals_host_on_gpu():
    a = gen.algebraic_decay(3000, seed=0)
    b = D.algebraic_decay(3000, seed=0, device="cuda").cpu().numpy()
    assert np.array_equal(a, b)
