"""Pins for the kernel of Eq. 10 with the self-cell term of Eq. 13 (Fig. 4
layout): the closed-form constant against cubature and the uniform-box
potential, and the symmetries of the kernel and its spectrum."""
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import SELF_TERM_C, green_kernel, green_spectrum
from oracle.green import circular_offsets
from tests.analytic import box_integral

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


def test_self_term_matches_golden():
    g = read_golden("self_term.txt")
    assert abs(SELF_TERM_C - g["C"]) < 1e-15


def test_self_term_by_face_quadrature():
    # integral of 1/r over the unit cube = 6 pyramids; each pyramid over a face at
    # distance h = 1/2 contributes (h / 2) * integral over the face of dA / |q|.
    f = lambda y, z: 1.0 / math.sqrt(0.25 + y * y + z * z)
    face, err = integrate.dblquad(f, -0.5, 0.5, -0.5, 0.5, epsabs=1e-13, epsrel=1e-13)
    assert abs(6 * 0.25 * face - SELF_TERM_C) < 1e-12


def test_self_term_by_midpoint_cubature_converges():
    errs = []
    for n in (40, 80):
        h = 1.0 / n
        c = -0.5 + (np.arange(n) + 0.5) * h
        x, y, z = np.meshgrid(c, c, c, indexing="ij")
        errs.append(abs(np.sum(1.0 / np.sqrt(x * x + y * y + z * z)) * h ** 3 - SELF_TERM_C))
    # midpoint rule on a 1/r singularity: error shrinks as the grid refines
    assert errs[1] < errs[0] and errs[1] < 2e-3


def test_box_formula_reduces_to_self_term_and_far_field():
    assert abs(box_integral(0, 0, 0, -.5, .5, -.5, .5, -.5, .5) - SELF_TERM_C) < 1e-13
    # far away a unit cube acts like a point mass, with the quadrupole vanishing
    # for a cube: error ~ r^-5
    for p in [(10.0, 0, 0), (6.0, 5.0, -4.0)]:
        r = math.sqrt(sum(v * v for v in p))
        assert abs(box_integral(*p, -.5, .5, -.5, .5, -.5, .5) - 1.0 / r) < 2e-5 / r
    # off-centre point inside the cube against brute-force cubature
    p = (0.2, -0.1, 0.3)
    n = 60
    h = 1.0 / n
    c = -0.5 + (np.arange(n) + 0.5) * h
    x, y, z = np.meshgrid(c, c, c, indexing="ij")
    cub = np.sum(1.0 / np.sqrt((x - p[0]) ** 2 + (y - p[1]) ** 2 + (z - p[2]) ** 2)) * h ** 3
    assert abs(box_integral(*p, -.5, .5, -.5, .5, -.5, .5) - cub) < 3e-3


def test_circular_layout():
    assert list(circular_offsets(4)) == [0, 1, 2, 3, 4, -3, -2, -1]


def test_kernel_values_and_symmetry():
    N = 4
    g = green_kernel(N)
    assert g[0, 0, 0] == SELF_TERM_C
    assert g[0, 0, 1] == 1.0 and g[0, 0, 7] == 1.0
    assert abs(g[1, 2, 3] - 1 / math.sqrt(14)) < 1e-16
    assert abs(g[7, 6, 5] - 1 / math.sqrt(14)) < 1e-16   # offsets (-1,-2,-3)
    assert np.array_equal(g, np.transpose(g, (1, 0, 2)))
    assert np.array_equal(g, np.transpose(g, (2, 1, 0)))
    # reflection j -> P - j
    P = 2 * N
    ref = g[(-np.arange(P)) % P][:, (-np.arange(P)) % P][:, :, (-np.arange(P)) % P]
    assert np.array_equal(g, ref)


@pytest.mark.parametrize("N", [4, 8])
def test_spectrum_real_even_and_dct(N):
    S = green_spectrum(N)
    assert np.max(np.abs(S.imag)) <= 1e-13 * np.max(np.abs(S.real))
    P = 2 * N
    Sr = S.real
    flip = (-np.arange(P)) % P
    assert np.allclose(Sr, Sr[flip][:, flip][:, :, flip], rtol=0, atol=1e-12)
    # the transform of a real even kernel is a 3-D DCT-I of its octant:
    # S(k) = sum_{j in [0, N]^3} w(j) g(j) prod cos(2 pi k j / P),
    # w = 1 at j in {0, N} and 2 otherwise, per axis.
    g = green_kernel(N)[: N + 1, : N + 1, : N + 1]
    j = np.arange(N + 1)
    w = np.where((j == 0) | (j == N), 1.0, 2.0)
    k = np.arange(N + 1)
    Cm = np.cos(2 * np.pi * np.outer(k, j) / P) * w[None, :]
    dct = np.einsum("az,by,cx,zyx->abc", Cm, Cm, Cm, g)
    assert np.allclose(Sr[: N + 1, : N + 1, : N + 1], dct, rtol=0, atol=1e-11)


def test_vectorised_box_formula_matches_the_scalar_one():
    from tests.analytic import box_integral_grid
    rng = np.random.default_rng(4)
    pts = rng.uniform(-1.2, 1.2, (40, 3))
    pts[0] = 0.0
    pts[1] = (0.5, 0.0, 0.25)       # on a face
    got = box_integral_grid(pts[:, 0], pts[:, 1], pts[:, 2], 0.5)
    for p, g in zip(pts, got):
        assert abs(g - box_integral(*p, -.5, .5, -.5, .5, -.5, .5)) < 1e-12 * max(1.0, abs(g))
