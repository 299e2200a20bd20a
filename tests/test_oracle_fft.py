"""Pins for the oracle's own FFT: the DFT definition, a library FFT, and the
transform's textbook identities."""
import numpy as np
import pytest

from oracle import fft_axis, fft3, ifft3


def dft_definition(x):
    n = len(x)
    j = np.arange(n)
    W = np.exp(-2j * np.pi * np.outer(j, j) / n)
    return W @ x


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64])
def test_matches_dft_definition(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = dft_definition(x)
    got = fft_axis(x)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_matches_library_fft_each_axis(axis):
    rng = np.random.default_rng(7)
    x = rng.standard_normal((8, 16, 32)) + 1j * rng.standard_normal((8, 16, 32))
    ref = np.fft.fft(x, axis=axis)
    assert np.allclose(fft_axis(x, axis), ref, rtol=0, atol=1e-12)
    ref_i = np.fft.ifft(x, axis=axis)
    assert np.allclose(fft_axis(x, axis, inverse=True), ref_i, rtol=0, atol=1e-14)


def test_3d_matches_library_and_round_trips():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((16, 16, 16)) + 1j * rng.standard_normal((16, 16, 16))
    X = fft3(x)
    assert np.allclose(X, np.fft.fftn(x), rtol=0, atol=1e-11)
    assert np.allclose(ifft3(X), x, rtol=0, atol=1e-14)


def test_identities():
    n = 32
    delta = np.zeros(n, complex)
    delta[0] = 1
    assert np.allclose(fft_axis(delta), np.ones(n))
    assert np.allclose(fft_axis(np.ones(n)), n * delta)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(n) + 0j
    # shift theorem: x[j - s] <-> X[k] exp(-2 pi i k s / n)
    s = 5
    k = np.arange(n)
    assert np.allclose(fft_axis(np.roll(x, s)), fft_axis(x) * np.exp(-2j * np.pi * k * s / n))
    # Parseval
    X = fft_axis(x)
    assert np.isclose(np.sum(np.abs(x) ** 2), np.sum(np.abs(X) ** 2) / n)


def test_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        fft_axis(np.ones(12))
