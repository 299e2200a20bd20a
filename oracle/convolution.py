"""Isolated convolution and direct summation (oracle, float64).

Eq. 10: Phi_i = -G sum_j M_j calG(x_i - x_j), calG = 1/(dx |i - j|) for i != j
and C/dx for i == j (Eq. 13).

Sect. 3 / Fig. 4: the sum is evaluated with the convolution theorem (Eq. 11) on
the doubled domain: M is zero-padded from N^3 to (2N)^3 (regions 2-4 of Fig. 4
carry zero mass), transformed, multiplied by the transform of the rearranged
kernel, transformed back and cropped to the active N^3 block.  Zero padding
makes the result the isolated (non-periodic) sum exactly, up to rounding.

Test infrastructure only; see the package docstring.
"""
import numpy as np

from .fft import fft3, ifft3
from .green import SELF_TERM_C, green_kernel, green_spectrum


def isolated_convolution(M, dx, G=1.0, spectrum=None):
    """Phi = -G sum_j M_j calG(i - j) on an N^3 block of cells of side dx.

    ``M`` is the cell-mass array (N, N, N) indexed [z, y, x].  ``spectrum`` is the
    unit-cell kernel transform on (2N)^3 (computed when not given).
    """
    M = np.asarray(M, dtype=np.float64)
    N = M.shape[0]
    if M.shape != (N, N, N):
        raise ValueError("mass block must be cubic")
    P = 2 * N
    if spectrum is None:
        spectrum = green_spectrum(N)
    padded = np.zeros((P, P, P), dtype=np.complex128)
    padded[:N, :N, :N] = M
    prod = fft3(padded) * spectrum
    conv = ifft3(prod)[:N, :N, :N].real
    return -G * conv / dx


def direct_sum(M, dx, G=1.0, kernel=None):
    """O(M^2) evaluation of Eq. 10 on an N^3 block (small N only).

    ``kernel``: optional unit-cell kernel on the (2N)^3 circular layout; when
    omitted the inverse distance and Eq. 13 self term are written out here
    directly from the cell-offset vectors.
    """
    M = np.asarray(M, dtype=np.float64)
    N = M.shape[0]
    idx = np.stack(np.meshgrid(np.arange(N), np.arange(N), np.arange(N),
                               indexing="ij"), axis=-1).reshape(-1, 3)
    d = idx[:, None, :] - idx[None, :, :]
    if kernel is None:
        r = np.sqrt((d.astype(np.float64) ** 2).sum(axis=-1))
        with np.errstate(divide="ignore"):
            g = np.where(r > 0, 1.0 / np.where(r > 0, r, 1.0), SELF_TERM_C)
    else:
        P = 2 * N
        g = kernel[d[..., 0] % P, d[..., 1] % P, d[..., 2] % P]
    phi = -G * (g @ M.reshape(-1)) / dx
    return phi.reshape(N, N, N)


def direct_sum_at(M, dx, G, targets):
    """Eq. 10 evaluated at given integer cell positions (any, also outside the
    block).  ``targets`` is (T, 3) of [z, y, x] cell coordinates in the same cell
    lattice as ``M``.  Returns (T,) potentials.  O(T * N^3).
    """
    M = np.asarray(M, dtype=np.float64)
    N = M.shape[0]
    zz, yy, xx = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    src = np.stack([zz.ravel(), yy.ravel(), xx.ravel()], axis=1).astype(np.float64)
    m = M.ravel()
    nz = m != 0.0
    src = src[nz]
    m = m[nz]
    out = np.empty(len(targets))
    for t, tgt in enumerate(np.asarray(targets, dtype=np.float64)):
        d = src - tgt[None, :]
        r = np.sqrt((d * d).sum(axis=1))
        self_mask = r == 0
        r_safe = np.where(self_mask, 1.0, r)
        g = np.where(self_mask, SELF_TERM_C, 1.0 / r_safe)
        out[t] = -G * float(np.dot(m, g)) / dx
    return out
