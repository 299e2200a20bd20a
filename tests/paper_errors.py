"""Relative potential errors (Eq. 7) of a nested solution against the analytic
potentials of the paper's test problems, over the composite mesh: every cell
of the finest level and the cells of each coarser level not covered by the
next finer one (each point of space counted once, at its finest level)."""
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


def composite_errors(w, phi):
    N, L = w.N, w.levels
    a, b = N // 4, 3 * N // 4
    errs = []
    for m in range(L):
        an = analytic_field(w, m)
        e = np.abs((phi[m] - an) / an)
        if m < L - 1:
            mask = np.ones((N, N, N), bool)
            mask[a:b, a:b, a:b] = False
            e = e[mask]
        errs.append(e.ravel())
    e = np.concatenate(errs)
    return {"max": float(e.max()), "mean": float(e.mean()), "std": float(e.std())}


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


def composite_accel_errors(w, g):
    """Eq. 7 errors of |g| (g: (levels, 3, N, N, N)) over the composite mesh."""
    N, L = w.N, w.levels
    a, b = N // 4, 3 * N // 4
    errs = []
    for m in range(L):
        gan = np.sqrt(sum(v * v for v in analytic_accel(w, m)))
        gnum = np.sqrt((g[m] ** 2).sum(axis=0))
        e = np.abs((gnum - gan) / gan)
        if m < L - 1:
            mask = np.ones((N, N, N), bool)
            mask[a:b, a:b, a:b] = False
            e = e[mask]
        errs.append(e.ravel())
    e = np.concatenate(errs)
    return {"max": float(e.max()), "mean": float(e.mean()), "std": float(e.std())}
