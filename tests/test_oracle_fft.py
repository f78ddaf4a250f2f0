"""Pins for the oracle's own FFT: the O(n^2) DFT definition, closed forms, and
numpy.fft as an independent library check."""
import numpy as np
import pytest

import oracle


def _cvec(n, seed):
    g = np.random.default_rng(seed)
    return g.normal(size=n) + 1j * g.normal(size=n)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 3, 6, 12, 24, 48, 96])
@pytest.mark.parametrize("inverse", [False, True])
def test_fft_matches_dft_definition(n, inverse):
    x = _cvec(n, n)
    a = oracle.fft1d(x, inverse)
    b = oracle.dft1d(x, inverse)
    assert np.abs(a - b).max() <= 1e-13 * max(1.0, np.abs(b).max())


@pytest.mark.parametrize("n", [2, 16, 256, 1024, 12, 48, 96, 384])
def test_fft_matches_numpy(n):
    x = _cvec(n, 100 + n)
    assert np.allclose(oracle.fft1d(x), np.fft.fft(x), rtol=0, atol=1e-12 * np.sqrt(n))
    assert np.allclose(oracle.fft1d(x, True), np.fft.ifft(x) * n, rtol=0, atol=1e-12 * np.sqrt(n))


def test_fft_closed_forms():
    n = 64
    delta = np.zeros(n, complex)
    delta[0] = 1
    assert np.abs(oracle.fft1d(delta) - 1).max() < 1e-15
    ones = np.ones(n, complex)
    f = oracle.fft1d(ones)
    assert abs(f[0] - n) < 1e-12 and np.abs(f[1:]).max() < 1e-12
    # a pure cosine at bin k0 puts n/2 at bins +-k0 and nothing elsewhere
    k0 = 5
    c = np.cos(2 * np.pi * k0 * np.arange(n) / n).astype(complex)
    f = oracle.fft1d(c)
    expect = np.zeros(n, complex)
    expect[k0] = expect[n - k0] = n / 2
    assert np.abs(f - expect).max() < 1e-12
    # a shifted delta gives the linear phase exp(-2 pi i k s / n)
    s = 3
    sd = np.zeros(n, complex)
    sd[s] = 1
    assert np.abs(oracle.fft1d(sd) - np.exp(-2j * np.pi * np.arange(n) * s / n)).max() < 1e-14


def test_fft_roundtrip_and_parseval():
    x = _cvec(256, 7)
    y = oracle.fft1d(x)
    assert np.abs(oracle.fft1d(y, True) / 256 - x).max() < 1e-14
    assert abs(np.vdot(y, y).real - 256 * np.vdot(x, x).real) < 1e-10 * np.vdot(y, y).real


@pytest.mark.parametrize("shape", [(8, 16), (64, 64), (32, 4), (48, 24), (96, 32)])
def test_fft2d_matches_numpy(shape):
    g = np.random.default_rng(1)
    x = g.normal(size=shape) + 1j * g.normal(size=shape)
    assert np.allclose(oracle.fft2d(x), np.fft.fft2(x), rtol=0, atol=1e-11)
    assert np.allclose(oracle.fft2d(x, True), np.fft.ifft2(x) * x.size, rtol=0, atol=1e-11)


def test_fft3d_matches_numpy():
    g = np.random.default_rng(2)
    x = g.normal(size=(8, 16, 4)) + 1j * g.normal(size=(8, 16, 4))
    assert np.allclose(oracle.fft3d(x), np.fft.fftn(x), rtol=0, atol=1e-11)


@pytest.mark.parametrize("n", [10, 18, 20, 7])
def test_fft_rejects_lengths_other_than_two_powers_times_one_or_three(n):
    with pytest.raises(ValueError):
        oracle.fft1d(np.ones(n, complex))
