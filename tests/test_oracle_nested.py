"""Pins for the nested decomposition of Sect. 4 (Eq. 14): geometry,
restriction, interpolation, special cases that reduce to one convolution or to
direct summation, analytic potentials, convergence order and invariants."""
import math

import numpy as np
import pytest

import oracle
from oracle import (Geometry, direct_sum, isolated_convolution, nested_potential_at,
                    restrict, solve, solve_components, trilinear_to_level)
from oracle.nested import interp_coords
from paper_2301_06763_gb300 import workloads as wl
from tests import analytic


def test_geometry_nesting():
    g = Geometry(3, 8, 0.1)
    for m in range(2):
        c, f = g.centres(m), g.centres(m + 1)
        a, b = g.covered
        # the two level-(m+1) cells inside level-m cell a + j straddle its centre
        for j in range(b - a):
            assert math.isclose(0.5 * (f[2 * j] + f[2 * j + 1]), c[a + j], abs_tol=1e-15)
        # level m+1 spans exactly the covered range of level m
        assert math.isclose(f[0] - g.dx(m + 1) / 2, c[a] - g.dx(m) / 2, abs_tol=1e-15)
        assert math.isclose(f[-1] + g.dx(m + 1) / 2, c[b - 1] + g.dx(m) / 2, abs_tol=1e-15)


@pytest.mark.parametrize("k,n", [(0, 1), (0, 2), (1, 3), (0, 4)])
def test_interp_coords_match_physical_coordinates(k, n):
    g = Geometry(5, 16, 0.37)
    u = interp_coords(16, k, n)
    phys = (g.centres(n) - g.centres(k)[0]) / g.dx(k)
    assert np.allclose(u, phys, rtol=0, atol=1e-12)


def test_trilinear_exact_for_multilinear_fields():
    N = 8
    g = Geometry(3, N, 1.0)
    for k, n in [(0, 1), (0, 2), (1, 2)]:
        ck, cn = g.centres(k), g.centres(n)
        f = lambda z, y, x: 1.5 + 2 * x - 3 * y + 0.5 * z + 0.25 * x * y * z - x * z
        Z, Y, X = np.meshgrid(ck, ck, ck, indexing="ij")
        Zn, Yn, Xn = np.meshgrid(cn, cn, cn, indexing="ij")
        got = trilinear_to_level(f(Z, Y, X), N, k, n)
        assert np.allclose(got, f(Zn, Yn, Xn), rtol=0, atol=1e-12)


def test_trilinear_weights_one_level_down():
    # a fine centre sits a quarter coarse cell from its parent's centre on each
    # axis: the per-axis weights are 3/4 (parent) and 1/4 (neighbour)
    u = interp_coords(8, 0, 1)
    t = u - np.floor(u)
    assert set(np.round(t, 15)) == {0.25, 0.75}


def test_restriction_conserves_mass():
    N, L = 8, 3
    rho = wl.random_density(1, L, N)
    g = Geometry(L, N, 0.5)
    r = restrict(rho, N)
    a, b = g.covered

    def composite_mass(arr):
        tot = 0.0
        for m in range(L):
            w = arr[m] * g.dx(m) ** 3
            if m < L - 1:
                w = w.copy()
                w[a:b, a:b, a:b] = 0
            tot += w.sum()
        return tot

    # the composite mesh's mass is unchanged, and every level carries all of it
    # that lies inside its own domain
    assert math.isclose(composite_mass(r), composite_mass(rho), rel_tol=1e-14)
    total = composite_mass(rho)
    assert math.isclose(r[0].sum() * g.dx(0) ** 3, total, rel_tol=1e-14)
    # the finest level is untouched
    assert np.array_equal(r[-1], rho[-1])


def test_single_level_is_plain_convolution():
    N = 8
    rho = wl.random_density(2, 1, N)
    got = solve(rho, N, 0.125)
    ref = direct_sum(rho[0] * 0.125 ** 3, 0.125)
    assert np.max(np.abs(got[0] - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_mass_only_inside_finest_level():
    # nothing outside level 1: Phi(Omega^1) is the plain fine-grid sum and the
    # coarse grid sees the restricted (2^3-averaged) mass
    N, dx0 = 8, 0.25
    rho = np.zeros((2, N, N, N))
    rng = np.random.default_rng(3)
    rho[1] = rng.random((N, N, N))
    out = solve(rho, N, dx0)
    fine = direct_sum(rho[1] * (dx0 / 2) ** 3, dx0 / 2)
    assert np.max(np.abs(out[1] - fine)) <= 1e-13 * np.max(np.abs(fine))
    coarse_rho = np.zeros((N, N, N))
    coarse_rho[2:6, 2:6, 2:6] = rho[1].reshape(4, 2, 4, 2, 4, 2).mean(axis=(1, 3, 5))
    coarse = direct_sum(coarse_rho * dx0 ** 3, dx0)
    assert np.max(np.abs(out[0] - coarse)) <= 1e-13 * np.max(np.abs(coarse))


@pytest.mark.parametrize("interp", ["trilinear", "diagonal"])
def test_mass_only_outside_fine_level(interp):
    # nothing inside level 1: Phi(Omega^1) is the interpolation of the exact
    # coarse sum (tensor-product linear, or the Eqs. 3-6 diagonal rule)
    from oracle.nested import diagonal_to_next
    N, dx0 = 8, 0.25
    rng = np.random.default_rng(4)
    rho = np.zeros((2, N, N, N))
    rho[0] = rng.random((N, N, N))
    rho[0, 2:6, 2:6, 2:6] = 0.0
    out = solve(rho, N, dx0, interp=interp)
    coarse = direct_sum(rho[0] * dx0 ** 3, dx0)
    assert np.max(np.abs(out[0] - coarse)) <= 1e-13 * np.max(np.abs(coarse))
    fine = trilinear_to_level(coarse, N, 0, 1) if interp == "trilinear" else diagonal_to_next(coarse, N)
    assert np.max(np.abs(out[1] - fine)) <= 1e-13 * np.max(np.abs(fine))


@pytest.mark.parametrize("L,method", [(2, "original"), (3, "original"), (2, "dipole"),
                                      (3, "dipole")])
def test_fft_route_equals_direct_route(L, method):
    N, dx0 = 8, 1.0 / 8
    rho = wl.random_density(10 + L, L, N)
    out = solve(rho, N, dx0, method=method, interp="trilinear")
    rng = np.random.default_rng(0)
    samples = [(n, *map(int, rng.integers(0, N, 3))) for n in range(L) for _ in range(4)]
    samples += [(L - 1, 0, 0, 0), (0, N - 1, N - 1, N - 1), (L - 1, 3, 4, 4)]
    ref = nested_potential_at(rho, N, dx0, samples, method=method, interp="trilinear")
    got = np.array([out[s] for s in samples])
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(out))


def test_plummer_analytic():
    w = wl.config_small()
    rho = w.rho()
    out = solve(rho, w.N, w.dx0)
    errs = []
    for m in range(w.levels):
        c = wl.level_centres(w.N, w.dx0, m)
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        an = analytic.plummer(np.sqrt(X * X + Y * Y + Z * Z), 1.0, 0.05)
        errs.append(np.abs((out[m] - an) / an))
    # 16 cells per level with a scale of 0.8 coarse cells: under 10 % at the
    # unresolved coarse centre, a few per cent on the finer level, and the finer
    # level is better resolved than the coarse one
    assert errs[0].max() < 0.10 and errs[1].max() < 0.03
    assert errs[0].mean() < 0.01 and errs[1].mean() < errs[0].mean()


def poly_errors(N, L=3, R=0.2):
    w = wl.Workload("poly", L, N, 1.0 / N, [wl.PolySphere(1.0, R, (0.01, -0.02, 0.005))])
    out = solve(w.rho(), N, w.dx0)
    e = []
    for m in range(L):
        c = wl.level_centres(N, w.dx0, m)
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        r = np.sqrt((X - 0.01) ** 2 + (Y + 0.02) ** 2 + (Z - 0.005) ** 2)
        e.append(np.abs(out[m] - analytic.poly_sphere(r, 1.0, R)))
    allerr = np.concatenate([x.ravel() for x in e])
    return allerr.max(), allerr.mean()


def test_second_order_convergence():
    # smooth compact density crossing the level interfaces: Phi max and mean
    # errors converge at second order (Sect. 7 convergence test)
    # (at N = 8 the sphere spans under two coarse cells, so the maximum error is
    # still pre-asymptotic there; the mean already converges at order 2)
    (m8, a8), (m16, a16), (m32, a32) = [poly_errors(N) for N in (8, 16, 32)]
    assert math.log2(m16 / m32) > 1.75
    assert math.log2(a8 / a16) > 1.9 and math.log2(a16 / a32) > 1.9


def test_linearity_and_scaling():
    N, L = 8, 3
    r1 = wl.random_density(20, L, N)
    r2 = wl.random_density(21, L, N, positive=False)
    a = solve(2.0 * r1 - 0.5 * r2, N, 0.1)
    b = 2.0 * solve(r1, N, 0.1) - 0.5 * solve(r2, N, 0.1)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))
    # Phi scales with dx^2 at fixed density (M ~ dx^3, calG ~ 1/dx), and with G
    c = solve(r1, N, 0.3, G=2.5)
    d = solve(r1, N, 0.1)
    assert np.max(np.abs(c - 2.5 * 9.0 * d)) <= 1e-13 * np.max(np.abs(c))


@pytest.mark.parametrize("method", ["original", "dipole"])
def test_cube_symmetries(method):
    N, L = 8, 3
    rho = wl.random_density(30, L, N)
    base = solve(rho, N, 0.125, method=method)
    ops = [lambda a: np.transpose(a, (0, 2, 1, 3)),      # swap z, y
           lambda a: np.transpose(a, (0, 3, 2, 1)),      # swap z, x
           lambda a: a[:, :, :, ::-1],                   # mirror x
           lambda a: np.transpose(a[:, ::-1], (0, 2, 3, 1))]  # mirror z then rotate
    for op in ops:
        got = solve(np.ascontiguousarray(op(rho)), N, 0.125, method=method)
        assert np.max(np.abs(got - op(base))) <= 1e-13 * np.max(np.abs(base))


@pytest.mark.parametrize("L,method", [(2, "original"), (4, "original"), (3, "dipole")])
def test_diagonal_interp_fft_route_equals_direct_route(L, method):
    # the carried Eqs. 3-6 interpolation: FFT convolutions + whole-level
    # carries against direct sums + a per-cell recursion
    N, dx0 = 8, 1.0 / 8
    rho = wl.random_density(20 + L, L, N)
    out = solve(rho, N, dx0, method=method, interp="diagonal")
    rng = np.random.default_rng(1)
    samples = [(n, *map(int, rng.integers(0, N, 3))) for n in range(L) for _ in range(3)]
    samples += [(L - 1, 0, 0, 0), (L - 1, N - 1, 0, N - 1)]
    ref = nested_potential_at(rho, N, dx0, samples, method=method, interp="diagonal")
    got = np.array([out[s] for s in samples])
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(out))


def test_diagonal_rule_linear_exact_and_quadratic_error():
    # Eqs. 3-6 are linear interpolation along the cell diagonal at a quarter of
    # its length: exact for linear fields, and for a quadratic with Hessian H
    # the error is t(1-t)/2 d^T H d = (3/32) d^T H d, d = dx_k (s_x, s_y, s_z)
    from oracle.acceleration import ghost_index
    from oracle.nested import diagonal_to_next
    N, dx0 = 16, 0.3
    geo = Geometry(2, N, dx0)
    c0, c1 = geo.centres(0), geo.centres(1)
    Z, Y, X = np.meshgrid(c0, c0, c0, indexing="ij")
    Zf, Yf, Xf = np.meshgrid(c1, c1, c1, indexing="ij")
    lin = lambda x, y, z: 0.7 * x - 1.3 * y + 2.1 * z + 0.4
    assert np.allclose(diagonal_to_next(lin(X, Y, Z), N), lin(Xf, Yf, Zf), rtol=0, atol=1e-13)
    H = np.array([[2.0, 1.0, 0.5], [1.0, -3.0, 0.0], [0.5, 0.0, 1.5]])   # (x, y, z) order
    q = lambda x, y, z: 0.5 * (H[0, 0] * x * x + H[1, 1] * y * y + H[2, 2] * z * z) + \
        H[0, 1] * x * y + H[0, 2] * x * z + H[1, 2] * y * z
    err = diagonal_to_next(q(X, Y, Z), N) - q(Xf, Yf, Zf)
    _, s = ghost_index(N, np.arange(N))
    Sz, Sy, Sx = np.meshgrid(s, s, s, indexing="ij")
    d = dx0 * np.stack([Sx, Sy, Sz])
    dHd = np.einsum("i...,ij,j...->...", d, H, d)
    assert np.allclose(err, 3.0 / 32.0 * dHd, rtol=0, atol=1e-13)


def test_diagonal_interp_carries_linear_holes_exactly():
    # a potential linear in space on every hole grid is carried down any
    # number of levels unchanged (each step is exact for linear fields)
    from oracle.nested import diagonal_to_next
    N, L, dx0 = 8, 4, 0.5
    geo = Geometry(L, N, dx0)
    f = lambda n: (lambda c: np.meshgrid(c, c, c, indexing="ij"))(geo.centres(n))
    lin = lambda Z, Y, X: 1.1 * X + 0.3 * Y - 0.8 * Z
    carry = None
    for n in range(1, L):
        hole = lin(*f(n - 1))
        carry = diagonal_to_next(hole if carry is None else carry + hole, N)
        assert np.allclose(carry, n * lin(*f(n)), rtol=0, atol=1e-12)
