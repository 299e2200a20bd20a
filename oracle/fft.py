"""Own radix-2 FFT for the oracle (float64 / complex128).

The convolution theorem of Sect. 3 (Eq. 11) is applied with a discrete Fourier
transform.  This module writes that transform out as the textbook recursive
decimation-in-time Cooley-Tukey split: X[k] = E[k] + w^k O[k] and
X[k + n/2] = E[k] - w^k O[k], w = exp(-2 pi i / n), where E and O are the
transforms of the even- and odd-indexed samples.

Normalisation (the 1/sqrt(2K) prefactor of Eq. 11 is garbled in the source):
the forward transform is unnormalised and the inverse carries 1/n per axis, so
ifft(fft(x)) == x.  Only power-of-two lengths are supported.

Test infrastructure only; see the package docstring.
"""
import numpy as np


def _fft_last(x, sign):
    n = x.shape[-1]
    if n == 1:
        return x.copy()
    even = _fft_last(x[..., 0::2], sign)
    odd = _fft_last(x[..., 1::2], sign)
    w = np.exp(sign * 2j * np.pi * np.arange(n // 2) / n)
    t = w * odd
    return np.concatenate([even + t, even - t], axis=-1)


def fft_axis(x, axis=-1, inverse=False):
    """1-D DFT of ``x`` along ``axis``.

    forward: X[k] = sum_j x[j] exp(-2 pi i j k / n)
    inverse: x[j] = (1/n) sum_k X[k] exp(+2 pi i j k / n)
    """
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[axis]
    if n < 1 or (n & (n - 1)) != 0:
        raise ValueError("oracle FFT supports power-of-two lengths only, got %d" % n)
    y = np.ascontiguousarray(np.moveaxis(x, axis, -1))
    y = _fft_last(y, +1.0 if inverse else -1.0)
    if inverse:
        y = y / n
    return np.ascontiguousarray(np.moveaxis(y, -1, axis))


def fft3(x):
    """Unnormalised 3-D DFT over the last three axes."""
    y = x
    for ax in (-1, -2, -3):
        y = fft_axis(y, ax)
    return y


def ifft3(x):
    """Inverse 3-D DFT (1/n per axis) over the last three axes."""
    y = x
    for ax in (-1, -2, -3):
        y = fft_axis(y, ax, inverse=True)
    return y
