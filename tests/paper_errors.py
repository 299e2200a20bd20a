"""Relative errors (Eq. 7) of a nested solution's potential and acceleration
against the analytic fields of the paper's test problems, over the composite
mesh: every cell of the finest level and the cells of each coarser level not
covered by the next finer one (each point of space counted once, at its
finest level).  plane=True keeps only the x-z plane through the centre (the
cells at y = +dx_m/2 of every level), where the paper evaluates its errors
(Sect. 6)."""
import numpy as np

from paper_2301_06763_gb300 import workloads as wl
from tests import analytic


def analytic_field(w, m):
    c = wl.level_centres(w.N, w.dx0, m)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    comp = w.components[0]
    if isinstance(comp, wl.HomogeneousSpheroid):
        return analytic.oblate_spheroid(X, Y, Z, comp.a, comp.c, comp.rho)
    tot = 0.0
    for s in w.components:
        r = np.sqrt((X - s.centre[0]) ** 2 + (Y - s.centre[1]) ** 2 + (Z - s.centre[2]) ** 2)
        M = 4.0 / 3.0 * np.pi * s.radius ** 3 * s.rho
        tot = tot + analytic.uniform_sphere(r, M, s.radius)
    return tot


def analytic_accel(w, m):
    """(gx, gy, gz) of the test problem at the centres of level m."""
    c = wl.level_centres(w.N, w.dx0, m)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    comp = w.components[0]
    if isinstance(comp, wl.HomogeneousSpheroid):
        return analytic.oblate_spheroid_accel(X, Y, Z, comp.a, comp.c, comp.rho)
    tot = [0.0, 0.0, 0.0]
    for s in w.components:
        M = 4.0 / 3.0 * np.pi * s.radius ** 3 * s.rho
        g = analytic.sphere_accel(X - s.centre[0], Y - s.centre[1], Z - s.centre[2], M, s.radius)
        tot = [t + v for t, v in zip(tot, g)]
    return tuple(tot)


def _composite(w, per_level, plane):
    N, L = w.N, w.levels
    a, b = N // 4, 3 * N // 4
    errs = []
    for m in range(L):
        e = per_level(m)
        mask = np.ones((N, N, N), bool)
        if m < L - 1:
            mask[a:b, a:b, a:b] = False
        if plane:
            e, mask = e[:, N // 2, :], mask[:, N // 2, :]
        errs.append(e[mask].ravel())
    e = np.concatenate(errs)
    return {"max": float(e.max()), "mean": float(e.mean()), "std": float(e.std())}


def composite_errors(w, phi, plane=False):
    """Eq. 7 errors of Phi (phi: (levels, N, N, N))."""
    def per_level(m):
        an = analytic_field(w, m)
        return np.abs((phi[m] - an) / an)
    return _composite(w, per_level, plane)


def composite_accel_errors(w, g, plane=False):
    """Eq. 7 errors of |g| (g: (levels, 3, N, N, N))."""
    def per_level(m):
        gan = np.sqrt(sum(v * v for v in analytic_accel(w, m)))
        return np.abs((np.sqrt((g[m] ** 2).sum(axis=0)) - gan) / gan)
    return _composite(w, per_level, plane)
