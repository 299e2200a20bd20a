"""Pins for the oblate-spheroid potential used to reproduce the paper's
Table 3: the ellipsoid integral by quadrature, the sphere limit, the far field
and Poisson's equation inside."""
import math

import numpy as np
from scipy import integrate

from tests import analytic


def quad_potential(x, y, z, a, c):
    # -pi G rho a^2 c int_lam^inf (1 - sum x_i^2/(a_i^2+u)) du / D(u), G = rho = 1
    R2, z2 = x * x + y * y, z * z
    if R2 / a ** 2 + z2 / c ** 2 <= 1.0:
        lam = 0.0
    else:
        f = lambda l: R2 / (a * a + l) + z2 / (c * c + l) - 1.0
        lo, hi = 0.0, 1.0
        while f(hi) > 0:
            hi *= 2.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if f(mid) > 0 else (lo, mid)
        lam = 0.5 * (lo + hi)
    g = lambda u: (1.0 - R2 / (a * a + u) - z2 / (c * c + u)) / ((a * a + u) * math.sqrt(c * c + u))
    val, _ = integrate.quad(g, lam, np.inf, epsabs=1e-13, epsrel=1e-12, limit=400)
    return -math.pi * a * a * c * val


def test_matches_quadrature_inside_and_outside():
    rng = np.random.default_rng(0)
    for _ in range(40):
        p = rng.uniform(-2.0, 2.0, 3)
        got = analytic.oblate_spheroid(*p, a=1.0, c=0.5)
        assert abs(got - quad_potential(*p, 1.0, 0.5)) < 1e-9 * abs(got)


def test_sphere_limit_and_far_field():
    # c -> a: the uniform sphere; far away: -M/r, M = 4/3 pi a^2 c
    for r in (0.3, 0.99, 1.5, 4.0):
        got = analytic.oblate_spheroid(r / math.sqrt(3), r / math.sqrt(3), r / math.sqrt(3), 1.0, 0.99999)
        ref = analytic.uniform_sphere(r, 4.0 / 3.0 * math.pi, 1.0)
        assert abs(got - ref) < 2e-4 * abs(ref)
    M = 4.0 / 3.0 * math.pi * 0.5
    far = analytic.oblate_spheroid(300.0, 0.0, 0.0, 1.0, 0.5)
    assert abs(far + M / 300.0) < 1e-5 * M / 300.0


def test_poisson_equation_inside():
    # Laplacian = 4 pi G rho = 4 pi inside (finite differences of a quadratic)
    h = 1e-3
    p = np.array([0.2, -0.1, 0.15])
    lap = 0.0
    f0 = analytic.oblate_spheroid(*p, 1.0, 0.5)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        lap += (analytic.oblate_spheroid(*(p + e), 1.0, 0.5) - 2 * f0
                + analytic.oblate_spheroid(*(p - e), 1.0, 0.5)) / (h * h)
    assert abs(lap - 4 * math.pi) < 1e-4 * 4 * math.pi
