"""Pins for the oracle's own FFT: the O(N^2) DFT definition, an independent
library FFT, Parseval, and impulse <-> constant."""
import numpy as np
import pytest

import oracle

SIZES = [1, 2, 3, 4, 5, 6, 8, 9, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 512]


@pytest.mark.parametrize("n", SIZES)
def test_fft1d_matches_definition(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    # the plain definition written in the test itself
    m = np.arange(n)
    W = np.exp(-2j * np.pi * np.outer(m, m) / n)
    ref = W @ x
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(oracle.fft1d(x, -1) - ref).max() / scale < 1e-13
    assert np.abs(oracle.dft_naive(x, -1) - ref).max() / scale < 1e-13
    ref_inv = np.conj(W) @ x
    assert np.abs(oracle.fft1d(x, +1) - ref_inv).max() / scale < 1e-13


@pytest.mark.parametrize("shape", [(16, 8, 8), (12, 6, 6), (4, 3, 2), (1, 1, 8), (2, 5, 3)])
def test_fft3_matches_numpy_and_naive(shape):
    rng = np.random.default_rng(sum(shape))
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    got = oracle.fft3(a, -1)
    ref = np.fft.fftn(a)
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-13
    # axis-by-axis naive DFT
    b = a.copy()
    for ax in range(3):
        b = np.apply_along_axis(lambda v: oracle.dft_naive(v, -1), ax, b)
    assert np.abs(got - b).max() / np.abs(b).max() < 1e-13
    back = oracle.fft3(got, +1) / a.size
    assert np.abs(back - a).max() < 1e-13 * np.abs(a).max() * 10


def test_parseval_and_impulse():
    rng = np.random.default_rng(5)
    a = rng.standard_normal((24, 12, 16)) + 1j * rng.standard_normal((24, 12, 16))
    A = oracle.fft3(a, -1)
    assert abs(np.sum(np.abs(A) ** 2) - a.size * np.sum(np.abs(a) ** 2)) / np.sum(np.abs(A) ** 2) < 1e-13
    imp = np.zeros((8, 6, 4), complex)
    imp[0, 0, 0] = 1.0
    assert np.abs(oracle.fft3(imp, -1) - 1.0).max() < 1e-15
    const = np.ones((8, 6, 4), complex)
    C = oracle.fft3(const, -1)
    expect = np.zeros_like(C)
    expect[0, 0, 0] = const.size
    assert np.abs(C - expect).max() < 1e-12
    # shifted impulse -> pure phase ramp exp(-2 pi i m k / N)
    imp = np.zeros((1, 1, 12), complex)
    imp[0, 0, 5] = 1.0
    m = np.arange(12)
    assert np.abs(oracle.fft3(imp, -1)[0, 0] - np.exp(-2j * np.pi * 5 * m / 12)).max() < 1e-14


def test_angular_frequency_convention():
    # numpy fftfreq convention, the Nyquist bin negative
    for n, d in [(8, 0.5), (9, 2.0), (12, 1e-6), (2, 1.0)]:
        ref = 2 * np.pi * np.fft.fftfreq(n, d)
        got = np.array([oracle.angular_freq(m, n, d) for m in range(n)])
        assert np.allclose(got, ref, rtol=1e-15, atol=0)
