"""Pins for the isolated convolution of Sect. 3: brute-force direct summation of
Eq. 10, the point-mass special case, and the unused kernel entries."""
import math

import numpy as np
import pytest

from oracle import SELF_TERM_C, direct_sum, green_kernel, green_spectrum, isolated_convolution
from oracle.convolution import direct_sum_at


def pair_loop(M, dx, G):
    """Eq. 10 written as a plain double loop over cells (tiny N only)."""
    N = M.shape[0]
    cells = [(z, y, x) for z in range(N) for y in range(N) for x in range(N)]
    out = np.zeros_like(M)
    for (z, y, x) in cells:
        s = 0.0
        for (c, b, a) in cells:
            if (z, y, x) == (c, b, a):
                s += M[c, b, a] * SELF_TERM_C / dx
            else:
                s += M[c, b, a] / (dx * math.sqrt((z - c) ** 2 + (y - b) ** 2 + (x - a) ** 2))
        out[z, y, x] = -G * s
    return out


def test_direct_sum_matches_pair_loop():
    rng = np.random.default_rng(0)
    M = rng.random((3, 3, 3))
    assert np.allclose(direct_sum(M, 0.3, 2.0), pair_loop(M, 0.3, 2.0), rtol=1e-14, atol=0)


@pytest.mark.parametrize("N,dx,G", [(2, 1.0, 1.0), (4, 0.25, 1.0), (8, 0.013, 6.674e-8),
                                    (16, 1.0 / 16, 1.0)])
def test_fft_convolution_equals_direct_sum(N, dx, G):
    rng = np.random.default_rng(N)
    M = rng.random((N, N, N)) - 0.3
    ref = direct_sum(M, dx, G)
    got = isolated_convolution(M, dx, G)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_point_mass():
    N, dx, G, m = 8, 0.5, 1.0, 3.0
    M = np.zeros((N, N, N))
    src = (2, 5, 1)
    M[src] = m
    phi = isolated_convolution(M, dx, G)
    zz, yy, xx = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    r = dx * np.sqrt((zz - src[0]) ** 2 + (yy - src[1]) ** 2 + (xx - src[2]) ** 2)
    exp = -G * m / np.where(r > 0, r, 1.0)
    exp[src] = -G * m * SELF_TERM_C / dx
    assert np.max(np.abs(phi - exp)) <= 1e-13 * np.max(np.abs(exp))


def test_circular_kernel_lookup_matches_inverse_distance():
    N = 4
    rng = np.random.default_rng(5)
    M = rng.random((N, N, N))
    assert np.allclose(direct_sum(M, 1.0, 1.0, kernel=green_kernel(N)),
                       direct_sum(M, 1.0, 1.0), rtol=1e-15, atol=0)


def test_entries_at_offset_N_never_matter():
    N = 8
    rng = np.random.default_rng(9)
    M = rng.random((N, N, N))
    a = isolated_convolution(M, 0.1, 1.0, green_spectrum(N))
    b = isolated_convolution(M, 0.1, 1.0, green_spectrum(N, half_value=123.456))
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


def test_direct_sum_at_matches_block_sum_and_far_points():
    N = 4
    rng = np.random.default_rng(2)
    M = rng.random((N, N, N))
    full = direct_sum(M, 0.2, 1.0)
    tg = np.array([[0, 0, 0], [3, 1, 2], [1, 1, 1]])
    assert np.allclose(direct_sum_at(M, 0.2, 1.0, tg), full[tg[:, 0], tg[:, 1], tg[:, 2]],
                       rtol=1e-14)
    # a point far outside sees the total mass at the block's centre of mass
    far = np.array([[400.0, 1.5, 1.5]])
    com = np.array([np.sum(M * np.arange(N)[:, None, None]) / M.sum(), 1.5, 1.5])
    r = 0.2 * np.linalg.norm(far[0] - com)
    assert abs(direct_sum_at(M, 0.2, 1.0, far)[0] + M.sum() / r) < 1e-4 * M.sum() / r
