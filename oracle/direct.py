"""Nested potential at sampled cells by direct summation only (oracle).

A second route to the same quantity as ``nested.solve``: every component
potential that the assembly needs at the sampled cell (Eq. 14, or Eqs. 15 and
B.1-B.2) is evaluated by the plain sum of Eq. 10 over the component's masses,
with no Fourier transform.  The cost is O(samples * levels * 8 * N^3), so it can
check a few cells of meshes far too large for the FFT oracle.

Test infrastructure only; see the package docstring.
"""
import numpy as np

from .convolution import direct_sum_at
from .acceleration import ghost_index
from .nested import Geometry, interp_coords, level_masses, restrict


def nested_potential_at(rho, N, dx0, samples, G=1.0, method="original", interp="diagonal"):
    """Phi(Omega^n) at cells ``samples`` = iterable of (n, z, y, x).

    interp='diagonal' evaluates the carried hole term of the Eqs. 3-6 reading
    recursively: carry_n(i) = 3/4 S_{n-1}(c) + 1/4 S_{n-1}(c + s), with
    S_k = Phi^k_hole + carry_k and (c, s) the nearest coarse cell and the
    diagonal step of fine cell i, every Phi^k_hole value a direct sum."""
    rho = np.asarray(rho, dtype=np.float64)
    L = rho.shape[0]
    geom = Geometry(L, N, dx0)
    rho_r = restrict(rho, N)
    full_M, hole_M = level_masses(rho_r, geom)
    hole_cache, carry_cache = {}, {}

    def hole_at(k, cell):
        if cell not in hole_cache.setdefault(k, {}):
            hole_cache[k][cell] = direct_sum_at(hole_M[k], geom.dx(k), G, np.array([cell], float))[0]
        return hole_cache[k][cell]

    def carry_at(n, cell):
        if n == 0:
            return 0.0
        if (n, cell) not in carry_cache:
            cs = [ghost_index(N, i) for i in cell]
            p0 = tuple(int(c) for c, _ in cs)
            p1 = tuple(int(c + sg) for c, sg in cs)
            carry_cache[(n, cell)] = (0.75 * (hole_at(n - 1, p0) + carry_at(n - 1, p0))
                                      + 0.25 * (hole_at(n - 1, p1) + carry_at(n - 1, p1)))
        return carry_cache[(n, cell)]

    if interp not in ("trilinear", "diagonal"):
        raise ValueError("interp must be 'trilinear' or 'diagonal'")
    out = []
    for (n, z, y, x) in samples:
        cell = np.array([[z, y, x]], dtype=np.float64)
        if method == "original" or n == L - 1:
            val = direct_sum_at(full_M[n], geom.dx(n), G, cell)[0]
        elif method in ("dipole3", "dipole3_ds") and n < L - 2:
            # Eqs. B.3 and B.6: own hole grid, level n+1's ring (level n+2's
            # region emptied) on its doubled grid reduced by 2^3, and level
            # n+2 on its quadrupled grid reduced by 4^3, or summed directly
            # at the level-n centre
            val = direct_sum_at(hole_M[n], geom.dx(n), G, cell)[0]
            sub2 = [[2 * z + dz - N // 2, 2 * y + dy - N // 2, 2 * x + dx - N // 2]
                    for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]
            val += direct_sum_at(hole_M[n + 1], geom.dx(n + 1), G, np.array(sub2, float)).mean()
            M2 = rho_r[n + 2] * geom.dx(n + 2) ** 3
            if method == "dipole3":
                sub4 = [[4 * z + dz - 3 * N // 2, 4 * y + dy - 3 * N // 2, 4 * x + dx - 3 * N // 2]
                        for dz in range(4) for dy in range(4) for dx in range(4)]
                val += direct_sum_at(M2, geom.dx(n + 2), G, np.array(sub4, float)).mean()
            else:
                centre = [[4 * v + 1.5 - 1.5 * N for v in (z, y, x)]]
                val += direct_sum_at(M2, geom.dx(n + 2), G, np.array(centre, float))[0]
        elif method in ("dipole", "dipole3", "dipole3_ds"):
            val = direct_sum_at(hole_M[n], geom.dx(n), G, cell)[0]
            # doubled fine grid of level n+1: 2N cells spanning level n, fine
            # block at [N/2, 3N/2).  The 2^3 fine cells inside coarse cell
            # (z, y, x) sit at 2*(z,y,x) + {0,1}; in the fine block's own index
            # lattice that is 2*(z,y,x) + {0,1} - N/2.
            fine = []
            for dz in (0, 1):
                for dy in (0, 1):
                    for dx in (0, 1):
                        fine.append([2 * z + dz - N // 2, 2 * y + dy - N // 2,
                                     2 * x + dx - N // 2])
            rho_fine_M = rho_r[n + 1] * geom.dx(n + 1) ** 3
            val += direct_sum_at(rho_fine_M, geom.dx(n + 1), G, np.array(fine, float)).mean()
        else:
            raise ValueError("method must be 'original', 'dipole', 'dipole3' or 'dipole3_ds'")
        if interp == "diagonal":
            out.append(val + carry_at(n, (int(z), int(y), int(x))))
            continue
        for k in range(n):
            u = interp_coords(N, k, n)
            pts, wts = [], []
            for idx_axis, i in enumerate((z, y, x)):
                i0 = int(np.floor(u[i]))
                t = u[i] - i0
                pts.append((i0, i0 + 1))
                wts.append((1.0 - t, t))
            corners, weights = [], []
            for a in (0, 1):
                for b in (0, 1):
                    for c in (0, 1):
                        corners.append([pts[0][a], pts[1][b], pts[2][c]])
                        weights.append(wts[0][a] * wts[1][b] * wts[2][c])
            vals = direct_sum_at(hole_M[k], geom.dx(k), G, np.array(corners, float))
            val += float(np.dot(weights, vals))
        out.append(val)
    return np.array(out)
