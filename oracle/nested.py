"""Nested-mesh convolution method (oracle, float64): Sect. 4 and Sect. 7.

Geometry (Sect. 2, Fig. 1): level m = 0 (coarsest) ... L-1 (finest), each N^3
cells, level m of cell size dx_m = dx0 / 2^m and side N dx_m, all levels centred
on the origin.  Cell centres: x_i = -N dx_m / 2 + (i + 1/2) dx_m.  Level m+1
therefore occupies level-m cells [N/4, 3N/4) on every axis (the same offset as
ib = N/4 + i/2 + 1 in Eqs. 3-6).  Arrays are indexed [level, z, y, x].

Readings taken where the paper is silent (each listed in the design notes):
* Coarse covered cells carry the restriction of the finer level (the mean of
  the 2^3 children, swept finest -> coarsest), so the coarse grid sees the fine
  mass (Sect. 4, Sect. 7 "projected from the fine to the coarse grid").  The
  caller's coarse values there are ignored.
* Cell mass M = rho(centre) * dx^3.
* The interpolation of Fig. 6 (stripped from the source) has two readings:
  interp='diagonal' (default): the two-point rule of Eqs. 3-6 (3/4 of the
  nearest coarse centre plus 1/4 of its diagonal neighbour towards the fine
  centre), the only interpolation the paper prints; it spans one level, so
  the coarser holes are carried down level by level:
  carry_n = D(carry_{n-1} + Phi^{n-1}_hole), carry_1 = D(Phi^0_hole).
  interp='trilinear': tensor-product linear, from level k straight to level
  n (no cascade through intermediate levels).  The two give the same
  potential errors; the diagonal one reproduces the paper's acceleration
  errors (Table 4) and its first-order convergence of the max g error.
* The "reduction" of the doubled fine grid to the coarse grid (Sect. 7) is the
  mean of the 2^3 fine values in each coarse cell.
* Eq. B.1 writes the coarser-level sum with superscript m = n; it is read as
  m = k (the same sum as Eq. 14).

Test infrastructure only; see the package docstring.
"""
from dataclasses import dataclass

import numpy as np

from .acceleration import ghost_index
from .convolution import isolated_convolution
from .green import green_spectrum


@dataclass(frozen=True)
class Geometry:
    levels: int
    N: int
    dx0: float

    def __post_init__(self):
        if self.levels < 1:
            raise ValueError("levels must be >= 1")
        if self.N < 4 or self.N % 4 != 0:
            raise ValueError("N must be a multiple of 4")

    def dx(self, m):
        return self.dx0 / (2.0 ** m)

    def centres(self, m):
        """Cell-centre coordinates of level m along one axis."""
        dx = self.dx(m)
        return -self.N * dx / 2.0 + (np.arange(self.N) + 0.5) * dx

    @property
    def covered(self):
        """Half-open index range of level m covered by level m + 1."""
        return self.N // 4, 3 * self.N // 4


def restrict(rho, N):
    """Replace each level's covered cells by the 2^3 mean of the finer level.

    Swept from the finest level to the coarsest, so every covered coarse cell
    holds the mean of the finest data below it and the total mass
    sum_m sum_uncovered rho dx_m^3 is exactly that of the composite mesh.
    """
    rho = np.array(rho, dtype=np.float64, copy=True)
    L = rho.shape[0]
    a, b = N // 4, 3 * N // 4
    h = N // 2
    for m in range(L - 2, -1, -1):
        child = rho[m + 1]
        avg = child.reshape(h, 2, h, 2, h, 2).mean(axis=(1, 3, 5))
        rho[m, a:b, a:b, a:b] = avg
    return rho


def level_masses(rho_restricted, geom):
    """Full and hole mass arrays per level (Fig. 5).

    full[m] = rho_m dx_m^3 on all N^3 cells; hole[m] = the same with the cells
    covered by level m + 1 set to zero (Omega^m_hole); the finest level has no
    hole grid (None).
    """
    L, N = geom.levels, geom.N
    a, b = geom.covered
    full, hole = [], []
    for m in range(L):
        M = rho_restricted[m] * geom.dx(m) ** 3
        full.append(M)
        if m < L - 1:
            Mh = M.copy()
            Mh[a:b, a:b, a:b] = 0.0
            hole.append(Mh)
        else:
            hole.append(None)
    return full, hole


def interp_coords(N, k, n):
    """Level-k fractional index of each level-n cell centre along one axis.

    From the geometry above: u = (x_i^n - x_0^k) / dx_k
      = N/2 - N/(2r) + (i + 1/2)/r - 1/2,   r = 2^(n-k).
    Written in index space it is exact in binary floating point (dyadic).
    """
    r = 2.0 ** (n - k)
    i = np.arange(N, dtype=np.float64)
    return N / 2.0 - N / (2.0 * r) + (i + 0.5) / r - 0.5


def trilinear_to_level(phi_k, N, k, n):
    """Tensor-product linear interpolation of a level-k field to the level-n
    cell centres (n > k), the tilde operator of Eq. 14 (Fig. 6)."""
    u = interp_coords(N, k, n)
    i0 = np.floor(u).astype(np.int64)
    t = u - i0
    if i0.min() < 0 or i0.max() + 1 > N - 1:
        raise AssertionError("interpolation stencil leaves level k")
    out = np.zeros((N, N, N))
    for az in (0, 1):
        wz = t if az else 1.0 - t
        for ay in (0, 1):
            wy = t if ay else 1.0 - t
            for ax in (0, 1):
                wx = t if ax else 1.0 - t
                vals = phi_k[np.ix_(i0 + az, i0 + ay, i0 + ax)]
                out += wz[:, None, None] * wy[None, :, None] * wx[None, None, :] * vals
    return out


def diagonal_to_next(phi_k, N):
    """The Eqs. 3-6 rule at every cell centre of level k+1 from level k: on
    each axis the fine centre lies a quarter coarse cell from the nearest
    coarse centre c, towards c + s; the value is 3/4 phi(c) + 1/4 phi(c + s)
    with s the diagonal step (+-1 on every axis)."""
    c, s = ghost_index(N, np.arange(N))
    return 0.75 * phi_k[np.ix_(c, c, c)] + 0.25 * phi_k[np.ix_(c + s, c + s, c + s)]


def reduce_2x(fine):
    """Mean of the 2^3 fine values in each coarse cell (the Sect. 7 reduction)."""
    n = fine.shape[0] // 2
    return fine.reshape(n, 2, n, 2, n, 2).mean(axis=(1, 3, 5))


def _level_convolution(job):
    """One level convolution of `solve_components` (a module-level function so
    that a process pool can run it); the spectrum is built where it runs."""
    M, dx, G = job
    return isolated_convolution(M, dx, G)


def solve_components(rho, N, dx0, G=1.0, method="original", want=("full", "hole"), mapper=None):
    """Per-level component potentials of the decomposition.

    Returns a dict with 'full' (Phi^m on Omega^m), 'hole' (Phi^m_hole on
    Omega^m_hole, None for the finest level), 'dbl' (reduced Phi^{m+1}_dbl on
    level m, pairwise-dipole method only) and 'rho' (restricted densities).

    The level convolutions are independent of one another (Sect. 4); with
    `mapper` (a map-like callable, e.g. a process pool's map) they are
    evaluated through it, with the same arithmetic and the same results.
    """
    rho = np.asarray(rho, dtype=np.float64)
    L = rho.shape[0]
    geom = Geometry(L, N, dx0)
    if rho.shape != (L, N, N, N):
        raise ValueError("rho must be (levels, N, N, N)")
    rho_r = restrict(rho, N)
    full_M, hole_M = level_masses(rho_r, geom)
    out = {"rho": rho_r, "full": [None] * L, "hole": [None] * L, "dbl": [None] * L}
    jobs = []
    for m in range(L):
        if "full" in want and (method == "original" or m == L - 1):
            jobs.append(("full", m, full_M[m]))
        if hole_M[m] is not None:
            jobs.append(("hole", m, hole_M[m]))
    if mapper is None:
        spec = green_spectrum(N)
        res = [isolated_convolution(M, geom.dx(m), G, spec) for (_, m, M) in jobs]
    else:
        res = list(mapper(_level_convolution, [(M, geom.dx(m), G) for (_, m, M) in jobs]))
    for (kind, m, _), r in zip(jobs, res):
        out[kind][m] = r
    if method == "dipole":
        spec2 = green_spectrum(2 * N) if L > 1 else None
        for n in range(L - 1):
            out["dbl"][n] = reduce_2x(doubled_fine_potential(rho_r[n + 1], geom, n + 1, G, spec2))
    elif method != "original":
        raise ValueError("method must be 'original' or 'dipole'")
    return out


def doubled_fine_potential(rho_fine, geom, m, G=1.0, spectrum=None):
    """Phi^m_dbl of Sect. 7 / Fig. 16: level m's mass on a grid of level-m cells
    with twice as many cells per axis (2N), spanning level m-1.  The level-m
    block sits in cells [N/2, 3N/2); the rest carries zero mass.  Returns the
    potential on all (2N)^3 cells."""
    N = geom.N
    Mdbl = np.zeros((2 * N, 2 * N, 2 * N))
    a, b = N // 2, 3 * N // 2
    Mdbl[a:b, a:b, a:b] = rho_fine * geom.dx(m) ** 3
    return isolated_convolution(Mdbl, geom.dx(m), G, spectrum)


def doubled_hole_potential(rho_fine, geom, m, G=1.0, spectrum=None):
    """Phi^m_dbl,hole of Appendix B (Fig. App0): as `doubled_fine_potential`,
    with the cells of level m covered by level m+1 emptied, so that the
    finer levels' mass is not counted twice."""
    N = geom.N
    a, b = geom.covered
    M = rho_fine.copy()
    M[a:b, a:b, a:b] = 0.0
    return doubled_fine_potential(M, geom, m, G, spectrum)


def quadrupled_potential(rho_fine, geom, m, G=1.0, spectrum=None):
    """Phi^m_qdp of Appendix B (Fig. App0): level m's mass on a grid of
    level-m cells extended to the physical size of level m-2 (4N cells per
    axis); the level-m block sits in cells [3N/2, 5N/2), the rest carries zero
    mass.  Returns the potential on all (4N)^3 cells."""
    N = geom.N
    Mq = np.zeros((4 * N, 4 * N, 4 * N))
    a, b = 3 * N // 2, 5 * N // 2
    Mq[a:b, a:b, a:b] = rho_fine * geom.dx(m) ** 3
    return isolated_convolution(Mq, geom.dx(m), G, spectrum)


def reduce_4x(fine):
    """Mean of the 4^3 fine values in each coarse cell (Phi_qdp reduced two
    levels down)."""
    n = fine.shape[0] // 4
    return fine.reshape(n, 4, n, 4, n, 4).mean(axis=(1, 3, 5))


def direct_two_down(rho_fine, geom, m, G=1.0):
    """Eq. B.6: the potential of level m's mass at the cell centres of level
    m-2 by direct summation of the inverse distance between the centres,
    -G sum_j M_j / |x_i - x_j| (the centres never coincide).  O(N^6)."""
    N = geom.N
    cf, cc = geom.centres(m), geom.centres(m - 2)
    M = (rho_fine * geom.dx(m) ** 3).ravel()
    Z, Y, X = np.meshgrid(cf, cf, cf, indexing="ij")
    src = np.stack([Z.ravel(), Y.ravel(), X.ravel()], axis=1)
    nz = M != 0.0
    src, M = src[nz], M[nz]
    Zc, Yc, Xc = np.meshgrid(cc, cc, cc, indexing="ij")
    tgt = np.stack([Zc.ravel(), Yc.ravel(), Xc.ravel()], axis=1)
    out = np.empty(len(tgt))
    for i0 in range(0, len(tgt), 256):
        d = tgt[i0:i0 + 256, None, :] - src[None, :, :]
        out[i0:i0 + 256] = -G * (M[None, :] / np.sqrt((d * d).sum(axis=-1))).sum(axis=1)
    return out.reshape(N, N, N)


def triple_terms(rho_r, geom, G, quadrupled=True):
    """The two finer-level terms of Eq. B.3 for every level n < L-2:
    reduce_2x(Phi^{n+1}_dbl,hole) and either reduce_4x(Phi^{n+2}_qdp) or,
    with quadrupled=False, the direct sum of Eq. B.6 from level n+2."""
    L, N = geom.levels, geom.N
    spec2 = green_spectrum(2 * N)
    spec4 = green_spectrum(4 * N) if quadrupled else None
    dbl, two = [None] * L, [None] * L
    for n in range(L - 2):
        dbl[n] = reduce_2x(doubled_hole_potential(rho_r[n + 1], geom, n + 1, G, spec2))
        if quadrupled:
            two[n] = reduce_4x(quadrupled_potential(rho_r[n + 2], geom, n + 2, G, spec4))
        else:
            two[n] = direct_two_down(rho_r[n + 2], geom, n + 2, G)
    return dbl, two


def solve(rho, N, dx0, G=1.0, method="original", interp="diagonal", mapper=None):
    """Potential on every cell of every level, shape (levels, N, N, N).

    method='original' -- Eq. 14:
        Phi(Omega^n) = Phi^n + sum_{k<n} tilde Phi^k_hole.
    method='dipole'   -- pairwise dipole method, Eqs. 15 and B.1-B.2:
        Phi(Omega^n) = Phi^n_hole + tilde Phi^{n+1}_dbl + sum_{k<n} tilde Phi^k_hole
                       for n below the finest level,
        Phi(Omega^L) = Phi^L + sum_{k<L} tilde Phi^k_hole on the finest.
    method='dipole3'  -- dipole moments across three neighbouring levels,
        Eqs. B.3-B.5: for n < L-2 (0-based)
        Phi(Omega^n) = Phi^n_hole + tilde Phi^{n+1}_dbl,hole + tilde Phi^{n+2}_qdp
                       + sum_{k<n} tilde Phi^k_hole,
        level L-2 as in the pairwise method, the finest as in Eq. 14.
    method='dipole3_ds' -- the same with tilde Phi^{n+2}_qdp replaced by the
        direct sum of Eq. B.6.
    interp='trilinear' takes each tilde Phi^k_hole straight from level k;
    interp='diagonal' replaces the sum over k < n by the carried term carry_n
    (module docstring).  `mapper`: see `solve_components`.
    """
    rho = np.asarray(rho, dtype=np.float64)
    L = rho.shape[0]
    triple = method in ("dipole3", "dipole3_ds")
    comp = solve_components(rho, N, dx0, G, "dipole" if triple else method, mapper=mapper)
    if triple:
        dbl3, two = triple_terms(comp["rho"], Geometry(L, N, dx0), G, quadrupled=method == "dipole3")
    if interp not in ("trilinear", "diagonal"):
        raise ValueError("interp must be 'trilinear' or 'diagonal'")
    out = np.zeros((L, N, N, N))
    carry = None
    for n in range(L):
        if method == "original" or n == L - 1:
            phi = comp["full"][n].copy()
        elif triple and n < L - 2:
            phi = comp["hole"][n] + dbl3[n] + two[n]
        else:
            phi = comp["hole"][n] + comp["dbl"][n]
        if interp == "trilinear":
            for k in range(n):
                phi += trilinear_to_level(comp["hole"][k], N, k, n)
        elif n > 0:
            src = comp["hole"][n - 1] if carry is None else carry + comp["hole"][n - 1]
            carry = diagonal_to_next(src, N)
            phi += carry
        out[n] = phi
    return out
