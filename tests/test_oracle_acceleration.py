"""Pins for the acceleration rules (Eq. 8 stencil, Eqs. 3-6 ghost values,
Appendix A methods A and B): exactness for linear potentials, the paper's
printed index formulas, and the convergence orders Sect. 7 states for g."""
import math

import numpy as np
import pytest

import oracle
from oracle.acceleration import ghost_index
from paper_2301_06763_gb300 import workloads as wl
from tests import analytic


def level_field(f, L, N, dx0):
    out = np.empty((L, N, N, N))
    for m in range(L):
        c = wl.level_centres(N, dx0, m)
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        out[m] = f(X, Y, Z)
    return out


def test_linear_potential_gives_exact_constant_field():
    N, L, dx0 = 8, 3, 0.37
    phi = level_field(lambda x, y, z: 2.0 * x - 3.0 * y + 0.5 * z + 7.0, L, N, dx0)
    g = oracle.acceleration(phi, N, dx0)
    for comp, val in enumerate((-2.0, 3.0, -0.5)):
        assert np.allclose(g[:, comp], val, rtol=0, atol=1e-12)


def test_quadratic_exact_away_from_interfaces():
    N, L, dx0 = 16, 2, 0.25
    phi = level_field(lambda x, y, z: x * x + 2 * y * y - z * z + x * y, L, N, dx0)
    g = oracle.acceleration(phi, N, dx0)
    c = wl.level_centres(N, dx0, 1)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    inner = (slice(1, N - 1),) * 3
    assert np.allclose(g[1, 0][inner], -(2 * X + Y)[inner], atol=1e-12)
    assert np.allclose(g[1, 1][inner], -(4 * Y + X)[inner], atol=1e-12)
    assert np.allclose(g[1, 2][inner], (2 * Z)[inner], atol=1e-12)


@pytest.mark.parametrize("N", [8, 16, 64])
def test_ghost_indices_follow_the_printed_formula(N):
    # Eqs. 3-6 index the fine and coarse grids 1-based with one ghost layer
    # (index 1 is the ghost): the coarse partner of fine index k is
    # kb = N/4 + k/2 + 1 (integer division), and the diagonal partner is kb+1
    # when k is odd, kb-1 when k is even.  In 0-based active indices,
    # i = k - 2 and c = kb - 2.
    for k in range(1, N + 3):
        i = k - 2
        kb = N // 4 + k // 2 + 1
        c, s = ghost_index(N, i)
        assert int(c) == kb - 2
        assert int(s) == (1 if k % 2 else -1)
    # the ghost left of the fine grid pairs coarse N/4 - 1 (weight 3/4) with N/4
    assert ghost_index(N, -1) == (N // 4 - 1, 1)


def accel_errors(N, L=3, R=0.2):
    w = wl.Workload("poly", L, N, 1.0 / N, [wl.PolySphere(1.0, R, (0.01, -0.02, 0.005))])
    phi = oracle.solve(w.rho(), N, w.dx0)
    g = oracle.acceleration(phi, N, w.dx0)
    errs = []
    a, b = N // 4, 3 * N // 4
    for m in range(L):
        c = wl.level_centres(N, w.dx0, m)
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        r = np.sqrt((X - 0.01) ** 2 + (Y + 0.02) ** 2 + (Z - 0.005) ** 2)
        gan = analytic.poly_sphere_accel_radial(r, 1.0, R)
        e = np.abs(np.sqrt((g[m] ** 2).sum(axis=0)) - gan) / gan
        mask = np.ones((N, N, N), bool)
        if m < L - 1:
            mask[a:b, a:b, a:b] = False
        mask &= r > 2 * w.dx0 / 2 ** m            # |g| -> 0 at the centre
        errs.append(e[mask])
    e = np.concatenate(errs)
    return e.max(), e.mean()


def test_acceleration_convergence_orders():
    # Sect. 7: mean error of g converges at second order, its maximum (at the
    # grid interfaces, where the interpolation is linear) at first order
    (m1, a1), (m2, a2), (m3, a3) = [accel_errors(N) for N in (16, 32, 64)]
    assert math.log2(a2 / a3) > 1.6
    assert 0.6 < math.log2(m2 / m3) < 1.6


def test_quadratic_exact_on_the_outer_boundary():
    # the one-sided second-order differences of the coarsest level are exact
    # for a quadratic; the central ones too, away from the finer level
    N, L, dx0 = 8, 1, 0.3
    phi = level_field(lambda x, y, z: 3 * x * x - y * y + 2 * z * z - x * z + y, L, N, dx0)
    g = oracle.acceleration(phi, N, dx0)
    c = wl.level_centres(N, dx0, 0)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    assert np.allclose(g[0, 0], -(6 * X - Z), atol=1e-11)
    assert np.allclose(g[0, 1], -(-2 * Y + 1), atol=1e-11)
    assert np.allclose(g[0, 2], -(4 * Z - X), atol=1e-11)


def _num_grad(f, x, y, z, h=1e-5):
    return tuple(-(f(*(p + h * e)) - f(*(p - h * e))) / (2 * h)
                 for p in [np.array([x, y, z])] for e in np.eye(3))


@pytest.mark.parametrize("pt", [(0.1, 0.2, 0.05), (0.3, -0.4, 0.2), (1.5, 0.2, -0.9), (0.0, 0.0, 1.2),
                                (-0.7, 0.8, 0.0)])
def test_analytic_accelerations_are_minus_the_gradient(pt):
    # the closed-form g of the test problems against a central difference of
    # their own closed-form potentials, inside and outside the bodies
    a, c = 1.0, 0.5
    f = lambda x, y, z: float(analytic.oblate_spheroid(x, y, z, a, c))
    g = analytic.oblate_spheroid_accel(*pt, a, c)
    assert np.allclose([float(v) for v in g], _num_grad(f, *pt), rtol=1e-6, atol=1e-9)
    M, R = 2.0, 0.6
    f = lambda x, y, z: float(analytic.uniform_sphere(math.sqrt(x * x + y * y + z * z), M, R))
    g = analytic.sphere_accel(*pt, M, R)
    assert np.allclose([float(v) for v in g], _num_grad(f, *pt), rtol=1e-6, atol=1e-9)
    r = math.sqrt(sum(v * v for v in pt))
    h = 1e-5
    dphi = (analytic.poly_sphere(r + h, M, R) - analytic.poly_sphere(r - h, M, R)) / (2 * h)
    assert abs(float(analytic.poly_sphere_accel_radial(r, M, R)) - float(dphi)) <= 1e-6 * abs(float(dphi))
