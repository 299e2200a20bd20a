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


def _face_fluxes(phi, N, n, ax, sigma, hat):
    # coarse and fine gradients across one face of the covered block, along
    # +sigma, from the substituted coarse field `hat`
    a, b = N // 4, 3 * N // 4
    cl, cov = (a - 1, a) if sigma > 0 else (b, b - 1)
    fl, gl = (0, -1) if sigma > 0 else (N - 1, N)
    sel = lambda i: tuple(i if t == ax else slice(a, b) for t in range(3))
    coarse = hat[sel(cov)] - phi[n][sel(cl)]
    from oracle.acceleration import ghost_face
    phi_B = np.squeeze(ghost_face(hat, N, ax, gl), axis=ax)
    fine = np.take(phi[n + 1], fl, axis=ax) - phi_B
    h = N // 2
    return coarse, fine.reshape(h, 2, h, 2).mean(axis=(1, 3))


@pytest.mark.parametrize("ax,sigma", [(0, 1), (1, -1), (2, 1), (2, -1)])
def test_method_C_matches_fluxes_across_the_interface(ax, sigma):
    # the defining property (Appendix A, method C): after the iterations the
    # coarse gradient across each face of the covered block equals the mean
    # of the fine gradients across it, (V - Phi_C)/dx_n = mean (Phi_f - Phi_B)/dx_{n+1}
    from oracle.acceleration import virtual_values
    N, L = 16, 3
    phi = np.random.default_rng(5).standard_normal((L, N, N, N))
    for n in range(L - 1):
        hat = virtual_values(phi[n], phi[n + 1], N, ax, sigma, iters=60)
        coarse, fine = _face_fluxes(phi, N, n, ax, sigma, hat)
        assert np.allclose(coarse / 1.0, fine / 0.5, rtol=0, atol=1e-12 * np.abs(phi).max())


def test_method_C_iteration_converges():
    # each sweep halves the change (the virtual value of a face cell depends on
    # those of its four diagonal face neighbours with weight 1/8 each)
    from oracle.acceleration import virtual_values
    N = 16
    phi = np.random.default_rng(6).standard_normal((2, N, N, N))
    d = [np.abs(virtual_values(phi[0], phi[1], N, 1, 1, k + 1) - virtual_values(phi[0], phi[1], N, 1, 1, k)).max()
         for k in (4, 8, 12)]
    assert d[1] <= d[0] / 8 and d[2] <= d[1] / 8


def test_method_C_exact_for_linear_and_equal_to_B_away_from_interfaces():
    N, L, dx0 = 16, 3, 0.4
    phi = level_field(lambda x, y, z: -0.6 * x + 1.7 * y + 0.9 * z + 2.0, L, N, dx0)
    gC = oracle.acceleration(phi, N, dx0, coarse_side="C")
    for comp, val in enumerate((0.6, -1.7, -0.9)):
        assert np.allclose(gC[:, comp], val, rtol=0, atol=1e-11)
    # a generic field: B and C differ only on the cells next to an interface
    phi = np.random.default_rng(7).standard_normal((L, N, N, N))
    gB = oracle.acceleration(phi, N, dx0)
    gC = oracle.acceleration(phi, N, dx0, coarse_side="C")
    a, b = N // 4, 3 * N // 4
    touched = np.zeros((L, N, N, N), bool)
    for n in range(L):
        if n > 0:       # fine side: boundary layers
            touched[n, [0, -1], :, :] = True
            touched[n, :, [0, -1], :] = True
            touched[n, :, :, [0, -1]] = True
        if n < L - 1:   # coarse side: the layers around the covered block
            touched[n, a - 1:b + 1, a - 1:b + 1, a - 1:b + 1] = True
            touched[n, a:b, a:b, a:b] = False
    diff = np.any(gB != gC, axis=1)
    assert not np.any(diff & ~touched)
    assert np.any(diff & touched)
