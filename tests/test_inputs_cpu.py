"""The counter-based input generator (ftk_inputs.hashed_amplitudes): its
numpy and torch forms produce the same bits, and its mixing function is the
published splitmix64 finaliser. CPU only."""
import numpy as np
import pytest

from ftk_inputs import hashed_amplitudes


def test_splitmix64_first_output():
    """splitmix64 from state 0: first output 0xE220A8397B1DCDAF (the
    generator's published reference sequence). seed 0, index 0 hashes the
    counter 0, so its real part is that output's top 53 bits / 2^53 - 1/2."""
    a = hashed_amplitudes(np.array([0]), 0)[0]
    assert a.real == (0xE220A8397B1DCDAF >> 11) * 2.0 ** -53 - 0.5


def test_numpy_and_torch_forms_agree():
    torch = pytest.importorskip("torch")
    idx = np.concatenate([np.arange(64), np.random.default_rng(1).integers(0, 1 << 30, 4096),
                          [(1 << 30) - 1, (1 << 33) + 5]]).astype(np.int64)
    for seed in (0, 7, 12345):
        a = hashed_amplitudes(idx, seed)
        b = hashed_amplitudes(torch.from_numpy(idx), seed, xp=torch).numpy()
        assert np.array_equal(a.real, b[:, 0]) and np.array_equal(a.imag, b[:, 1])


def test_moments():
    """Uniform on [-1/2, 1/2) per component: mean 0, variance 1/12."""
    a = hashed_amplitudes(np.arange(1 << 16), 3)
    for c in (a.real, a.imag):
        assert abs(c.mean()) < 0.01 and abs(c.var() * 12 - 1) < 0.02
        assert c.min() >= -0.5 and c.max() < 0.5
