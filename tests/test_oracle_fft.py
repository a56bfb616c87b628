"""Pins of the oracle's radix-2 FFT and direct DFT (FFT / IFFT blocks of Fig. 2).

Checked against numpy's FFT (a library routine), Parseval, impulse and tone
special cases and the inverse-of-forward identity.
"""
import numpy as np
import pytest

import oracle

rng = np.random.default_rng(7)


@pytest.mark.parametrize("N", [1, 2, 4, 8, 64, 256, 2048, 4096, 16384])
def test_fft_matches_numpy(N):
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    ref = np.fft.fft(x)
    scale = np.abs(ref).max()
    assert np.abs(oracle.fft(x) - ref).max() <= 1e-12 * max(scale, 1.0) * np.log2(max(N, 2))
    refi = np.fft.ifft(x)
    assert np.abs(oracle.fft(x, inverse=True) - refi).max() <= 1e-12 * max(np.abs(refi).max(), 1e-3) * np.log2(max(N, 2))


@pytest.mark.parametrize("N", [3, 16, 100, 1024, 4096])
def test_dft_matches_numpy(N):
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    ref = np.fft.fft(x)
    assert np.abs(oracle.dft(x) - ref).max() <= 1e-12 * np.abs(ref).max() * np.sqrt(N)
    assert np.abs(oracle.dft(x, inverse=True) - np.fft.ifft(x)).max() <= 1e-12 * np.sqrt(N)


@pytest.mark.parametrize("N", [512, 4096])
def test_fft_equals_direct_dft(N):
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    a = oracle.fft(x)
    b = oracle.dft(x)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max() * np.sqrt(N)


def test_parseval():
    N = 8192
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    X = oracle.fft(x)
    assert abs((np.abs(X) ** 2).sum() / N - (np.abs(x) ** 2).sum()) <= 1e-10 * (np.abs(x) ** 2).sum()


def test_impulse_and_tone():
    N = 2048
    d = np.zeros(N, complex)
    d[0] = 1.0
    np.testing.assert_allclose(oracle.fft(d), np.ones(N), atol=1e-14)
    k0 = 37
    tone = np.exp(2j * np.pi * k0 * np.arange(N) / N)
    X = oracle.fft(tone)
    assert abs(X[k0] - N) < 1e-9
    X[k0] = 0
    assert np.abs(X).max() < 1e-9
    # a shifted impulse gives a pure linear phase
    d = np.zeros(N, complex)
    d[5] = 1.0
    np.testing.assert_allclose(oracle.fft(d), np.exp(-2j * np.pi * 5 * np.arange(N) / N), atol=1e-12)


def test_roundtrip():
    N = 4096
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    assert np.abs(oracle.fft(oracle.fft(x), inverse=True) - x).max() < 1e-13 * np.abs(x).max() * 12


def test_non_power_of_two_rejected():
    with pytest.raises(ValueError):
        oracle.fft(np.ones(12))
