"""Green's function of the discrete potential sum (oracle, float64).

Eq. 10 writes the cell potential as Phi_i = -G sum_j M_j * calG(x_i - x_j) with
calG the inverse distance between cell centres.  For a cell of side dx and an
integer offset d (in cells) calG = 1 / (dx |d|).

Self-cell term (Eq. 13, Sect. 3): with the density constant inside the cell, the
cell's own contribution is -G rho * integral over the cell of dV / r.  For a cube
of side dx that integral is dx^2 * C with the closed form
    C = 3 ln(2 + sqrt 3) - pi / 2 = 2.38007736...
(the analytic value the paper points to; tests pin it against cubature and
against the uniform-box potential formula).  Since M = rho dx^3 the self entry of
calG is C / dx.

Doubled, rearranged domain (Fig. 4, Sect. 3): the kernel lives on the (2N)^3
periodic domain with offsets laid out circularly, index j <-> offset j for
j <= N and j - 2N for j > N.  Reading: the entry at offset +N (index N on some
axis) is never used for source and target both inside the active N^3 block;
it is set to the plain inverse distance 1/|d| with d = +N on that axis.

All quantities here are for unit cell size (dx = 1); the convolution scales by
1/dx.  Test infrastructure only; see the package docstring.
"""
import math

import numpy as np

from .fft import fft3

SELF_TERM_C = 3.0 * math.log(2.0 + math.sqrt(3.0)) - math.pi / 2.0


def circular_offsets(N):
    """Offsets (in cells) along one axis of the doubled domain, Fig. 4."""
    P = 2 * N
    j = np.arange(P)
    return np.where(j <= N, j, j - P).astype(np.float64)


def green_kernel(N, half_value=None):
    """Unit-cell inverse-distance kernel on the (2N)^3 circular layout.

    ``half_value``: if given, every entry with offset +N on any axis is replaced
    by it (used by the test that shows those entries never matter).
    """
    d = circular_offsets(N)
    dz, dy, dx = np.meshgrid(d, d, d, indexing="ij")
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    with np.errstate(divide="ignore"):
        g = 1.0 / r
    g[0, 0, 0] = SELF_TERM_C
    if half_value is not None:
        P = 2 * N
        mask = np.zeros((P, P, P), dtype=bool)
        mask[N, :, :] = True
        mask[:, N, :] = True
        mask[:, :, N] = True
        g[mask] = half_value
    return g


def green_spectrum(N, half_value=None):
    """Forward 3-D DFT of ``green_kernel`` (complex128, full (2N)^3)."""
    return fft3(green_kernel(N, half_value).astype(np.complex128))
