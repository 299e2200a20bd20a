"""Pins for the pairwise-dipole ("modified") method of Sect. 7 and Appendix B
(Eqs. 15, B.1-B.2) and for its three-level extension (Eqs. B.3-B.6)."""
import numpy as np
import pytest

from oracle import nested, solve
from oracle.nested import doubled_fine_potential, Geometry
from oracle.convolution import direct_sum
from paper_2301_06763_gb300 import workloads as wl


def test_finest_level_identical_in_both_methods():
    N, L = 8, 3
    rho = wl.random_density(40, L, N)
    a = solve(rho, N, 0.125)
    b = solve(rho, N, 0.125, method="dipole")
    assert np.max(np.abs(a[-1] - b[-1])) <= 1e-13 * np.max(np.abs(a))


def test_doubled_grid_is_the_fine_block_sum_on_a_wider_lattice():
    # Phi_dbl on the 2N lattice equals the brute-force sum of Eq. 10 over the
    # fine block placed at [N/2, 3N/2)
    N = 4
    g = Geometry(2, N, 0.5)
    rng = np.random.default_rng(1)
    rho_f = rng.random((N, N, N))
    got = doubled_fine_potential(rho_f, g, 1)
    M = np.zeros((2 * N,) * 3)
    M[N // 2:3 * N // 2, N // 2:3 * N // 2, N // 2:3 * N // 2] = rho_f * g.dx(1) ** 3
    ref = direct_sum(M, g.dx(1))
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def electric_dipole(N=16, q=1.0):
    """+q and -q in two neighbouring finest cells that share one coarse cell,
    so they cancel exactly when restricted to the coarse grid (Fig. 15)."""
    dx0 = 1.0 / N
    rho = np.zeros((2, N, N, N))
    v = q / (dx0 / 2) ** 3
    c = N // 2
    rho[1, c, c, c] = v          # +q
    rho[1, c, c, c + 1] = -v     # -q, same parent coarse cell
    return rho, dx0


def test_dipole_cancels_on_coarse_grid_in_original_method():
    rho, dx0 = electric_dipole()
    out = solve(rho, 16, dx0)
    assert np.max(np.abs(out[0])) < 1e-12 * np.max(np.abs(out[1]))


def test_modified_method_restores_dipole_field_on_coarse_grid():
    N = 16
    rho, dx0 = electric_dipole(N)
    out = solve(rho, N, dx0, method="dipole")
    dxf = dx0 / 2
    c = wl.level_centres(N, dx0, 1)
    p_plus = np.array([c[N // 2], c[N // 2], c[N // 2]])
    p_minus = np.array([c[N // 2], c[N // 2], c[N // 2 + 1]])
    cc = wl.level_centres(N, dx0, 0)
    Z, Y, X = np.meshgrid(cc, cc, cc, indexing="ij")
    pos = np.stack([Z, Y, X], -1)
    exact = -(1.0 / np.linalg.norm(pos - p_plus, axis=-1)
              - 1.0 / np.linalg.norm(pos - p_minus, axis=-1))
    r = np.linalg.norm(pos - 0.5 * (p_plus + p_minus), axis=-1)
    far = r > 4 * dx0
    # the coarse value is the mean over the 2^3 fine cells of the coarse cell,
    # which differs from the centre value at O((dx/r)^2)
    err = np.abs(out[0][far] - exact[far])
    assert np.max(err / np.max(np.abs(exact[far]))) < 0.05
    assert np.corrcoef(out[0][far], exact[far])[0, 1] > 0.999


def test_modified_close_to_original_for_smooth_density():
    # Appendix C: on smooth densities the two methods barely differ.  Here the
    # Plummer core (scale 0.05) is unresolved on the 16^3 coarse level, so they
    # differ inside the covered region, where the modified method, which sees
    # the fine-level mass, is the closer one to the analytic potential.
    from tests import analytic
    w = wl.config_small()
    rho = w.rho()
    a = solve(rho, w.N, w.dx0)
    b = solve(rho, w.N, w.dx0, method="dipole")
    assert np.mean(np.abs(a - b) / np.abs(a)) < 1e-3
    c = wl.level_centres(w.N, w.dx0, 0)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    an = analytic.plummer(np.sqrt(X * X + Y * Y + Z * Z), 1.0, 0.05)
    err_a = np.abs(a[0] - an) / np.abs(an)
    err_b = np.abs(b[0] - an) / np.abs(an)
    assert err_b.max() < err_a.max() and err_b.mean() <= err_a.mean()


@pytest.mark.parametrize("method", ["dipole3", "dipole3_ds"])
def test_triple_fft_route_equals_direct_route(method):
    # Eqs. B.3-B.6: every term of the three-level dipole scheme by the FFT
    # convolutions (doubled and quadrupled grids) against direct sums at the
    # sub-cells (2^3 and 4^3 means) or, for Eq. B.6, at the coarse centres
    from oracle import nested_potential_at
    N, L, dx0 = 8, 4, 1.0 / 8
    rho = wl.random_density(31, L, N)
    out = solve(rho, N, dx0, method=method, interp="trilinear")
    rng = np.random.default_rng(2)
    samples = [(n, *map(int, rng.integers(0, N, 3))) for n in range(L) for _ in range(3)]
    samples += [(0, 0, 0, 0), (1, N - 1, 3, 4), (0, 3, 4, 4)]
    ref = nested_potential_at(rho, N, dx0, samples, method=method, interp="trilinear")
    got = np.array([out[s] for s in samples])
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(out))


def test_triple_scheme_keeps_a_dipole_two_levels_down():
    # Sect. 7 / Appendix B: a +-q pair inside one level-1 cell on the finest of
    # three levels.  The pairwise scheme sees the pair on level 0 only through
    # level 1's restricted (zero) mass, so level 0 gets nothing; the three-level
    # scheme reads the finest level on its quadrupled grid and level 0 gets the
    # dipole field of the pair.
    N, L, dx0 = 16, 3, 1.0
    rho = np.zeros((L, N, N, N))
    rho[2, 8, 8, 8], rho[2, 8, 8, 9] = 1.0, -1.0         # one level-1 cell: x = 8, 9 -> 4
    two = solve(rho, N, dx0, method="dipole")
    three = solve(rho, N, dx0, method="dipole3")
    ds = solve(rho, N, dx0, method="dipole3_ds")
    assert np.max(np.abs(two[0])) == 0.0
    # the point-dipole potential of the pair at the level-0 centres, away from it
    g = nested.Geometry(L, N, dx0)
    c0, c2 = g.centres(0), g.centres(2)
    Z, Y, X = np.meshgrid(c0, c0, c0, indexing="ij")
    m = g.dx(2) ** 3
    r1 = np.sqrt((X - c2[8]) ** 2 + (Y - c2[8]) ** 2 + (Z - c2[8]) ** 2)
    r2 = np.sqrt((X - c2[9]) ** 2 + (Y - c2[8]) ** 2 + (Z - c2[8]) ** 2)
    ref = -m / r1 + m / r2
    far = r1 > 3 * g.dx(0)
    for got in (three[0], ds[0]):
        assert np.corrcoef(got[far], ref[far])[0, 1] > 0.999
    # Eq. B.6 is the exact point-to-point sum: equal to the reference everywhere
    assert np.allclose(ds[0], ref, rtol=0, atol=1e-12 * np.abs(ref).max())
