"""Gravitational acceleration from the nested potential (oracle, float64).

g = -grad Phi by the central six-point stencil of Eq. 8 on every level (the
minus sign missing from Eq. 8 as printed is read as a typo: Appendix A writes
g = -(Phi_{i+1} - Phi_{i-1}) / (2 dx)).  Where the stencil leaves a level
(Sect. 2 and Appendix A, the "first, simple method" the paper uses):

* fine side (method A): a cell on the boundary of level n >= 1 takes the
  missing neighbour from a ghost value Phi_B interpolated from level n-1 by
  Eqs. 3-6: the ghost centre lies a quarter of a coarse cell from the nearest
  coarse centre c on each axis, and Phi_B = 3/4 Phi(c) + 1/4 Phi(c + s), s the
  diagonal step (+-1 per axis) towards the ghost centre;
* coarse side (method B): an uncovered cell of level n whose neighbour is
  covered by level n+1 takes for that neighbour the mean of its 2^3 children's
  potentials on level n+1 (the 2-D text averages 4 fine cells);
* coarse side (method C, coarse_side="C"): that neighbour takes instead a
  virtual value V chosen so that the coarse-grid gradient across the shared
  face, (V - Phi_C)/dx_n, equals the mean of the fine-grid gradients across
  the same face, (Phi_f - Phi_B)/dx_{n+1}, over the 2x2 fine cells f touching
  it, Phi_B being their Eqs. 3-6 ghost values.  The ghost values themselves
  read the coarse level at covered cells next to the face, so V is put back
  into Eqs. 3-6 and the two steps repeated (`iters` times, from V = the
  coarse level's own value there); the fine cells' ghosts (method A) then use
  the final substituted values as well;
* outer boundary of the coarsest level (the paper is silent): second-order
  one-sided differences.

Covered cells themselves use plain central differences of their own level.
Phi is the (levels, N, N, N) nested potential; the result is
(levels, 3, N, N, N) with components (gx, gy, gz) along the array axes
(2, 1, 0).  Test infrastructure only; see the package docstring.
"""
import numpy as np


def ghost_index(N, i):
    """Nearest level-(n-1) index c and diagonal step s of level-n cell-centre
    index i (i = -1 or N for a ghost), per axis: u = N/4 + (i + 1/2)/2 - 1/2
    = c + s/4 (s = +1 or -1)."""
    i = np.asarray(i)
    # u = (N/2 + i)/2 - 1/4: c = floor((N/2 + i)/2), s = +1 for odd i (N/2 is even)
    c = (N // 2 + i) // 2
    s = np.where(i % 2 == 1, 1, -1)
    return c, s


def ghost_face(phi_c, N, ax, side):
    """Eqs. 3-6 ghost values of level n for the face just outside index
    `side` (-1 or N) along array axis `ax`, from the level-(n-1) potential:
    an (N, N) array over the two other axes, as an N^3 slice shape."""
    idx = [np.arange(N)] * 3
    idx[ax] = np.array([side])
    cs, ss = zip(*(ghost_index(N, t) for t in idx))
    near = phi_c[np.ix_(cs[0], cs[1], cs[2])]
    diag = phi_c[np.ix_(cs[0] + ss[0], cs[1] + ss[1], cs[2] + ss[2])]
    return 0.75 * near + 0.25 * diag


def _face_layer(ax, i):
    """Index tuple selecting layer i of array axis ax."""
    sl = [slice(None)] * 3
    sl[ax] = i
    return tuple(sl)


def virtual_values(phi_c, phi_f, N, ax, sigma, iters):
    """Method C on one face of the covered block of level n (array axis ax;
    sigma = +1: the face at coarse index N/4 - 1 | N/4, sigma = -1: the face
    at 3N/4 - 1 | 3N/4).  Returns the level-n field hat_phi: phi_c with the
    covered cells next to the face replaced by the converged virtual values
    (their coarse-grid stand-ins seen through that face)."""
    a, b = N // 4, 3 * N // 4
    cl = a - 1 if sigma > 0 else b            # uncovered coarse layer C
    cov = cl + sigma                          # covered layer C'
    fl = 0 if sigma > 0 else N - 1            # fine layer touching the face
    ghost = -1 if sigma > 0 else N            # fine ghost layer across it
    dxr = 2.0                                 # dx_n / dx_{n+1}
    tang = [t for t in range(3) if t != ax]
    hat = phi_c.copy()
    inner = [slice(a, b)] * 3
    inner[ax] = cov
    inner = tuple(inner)
    cells = [slice(a, b)] * 3
    cells[ax] = cl
    cells = tuple(cells)
    for _ in range(iters):
        phi_B = ghost_face(hat, N, ax, ghost)                    # Eqs. 3-6, (N, N) over the fine face
        phi_B = np.squeeze(phi_B, axis=ax)
        fine = phi_f[_face_layer(ax, fl)]
        h = N // 2
        dfine = (fine - phi_B).reshape(h, 2, h, 2).mean(axis=(1, 3))
        # (V - Phi_C) / dx_n = mean (Phi_f - Phi_B) / dx_{n+1}, both along +sigma
        V = phi_c[cells] + dxr * dfine
        hat[inner] = V
    return hat


def _shift(p, ax, step):
    """p at index i + step along ax (edge values wrap and are replaced later)."""
    return np.roll(p, -step, axis=ax)


def acceleration(phi, N, dx0, coarse_side="B", iters=32):
    phi = np.asarray(phi, dtype=np.float64)
    L = phi.shape[0]
    a, b = N // 4, 3 * N // 4
    if coarse_side not in ("B", "C"):
        raise ValueError("coarse_side must be 'B' or 'C'")
    # method C: per interface and face, the coarse level with its virtual values
    hat = {}
    if coarse_side == "C":
        for n in range(L - 1):
            for ax in (0, 1, 2):
                for sigma in (1, -1):
                    hat[(n, ax, sigma)] = virtual_values(phi[n], phi[n + 1], N, ax, sigma, iters)
    g = np.zeros((L, 3, N, N, N))
    for n in range(L):
        dx = dx0 / 2.0 ** n
        p = phi[n]
        for comp, ax in enumerate((2, 1, 0)):
            plus, minus = _shift(p, ax, +1), _shift(p, ax, -1)
            sl_lo = [slice(None)] * 3
            sl_hi = [slice(None)] * 3
            sl_lo[ax] = slice(0, 1)
            sl_hi[ax] = slice(N - 1, N)
            if n < L - 1:
                if coarse_side == "B":
                    # method B: the covered block as the children's means
                    f = phi[n + 1]
                    h = N // 2
                    R = f.reshape(h, 2, h, 2, h, 2).mean(axis=(1, 3, 5))
                    # cells at index a-1 (neighbour a covered) and b (neighbour b-1)
                    for cell_i, nb_i, arr in ((a - 1, a, plus), (b, b - 1, minus)):
                        tgt = [slice(a, b)] * 3
                        tgt[ax] = slice(cell_i, cell_i + 1)
                        src = [slice(None)] * 3
                        src[ax] = slice(nb_i - a, nb_i - a + 1)
                        arr[tuple(tgt)] = R[tuple(src)]
                else:
                    # method C: the virtual values of the face
                    for cell_i, nb_i, arr, sigma in ((a - 1, a, plus, 1), (b, b - 1, minus, -1)):
                        tgt = [slice(a, b)] * 3
                        tgt[ax] = slice(cell_i, cell_i + 1)
                        src = [slice(a, b)] * 3
                        src[ax] = slice(nb_i, nb_i + 1)
                        arr[tuple(tgt)] = hat[(n, ax, sigma)][tuple(src)]
            d = (plus - minus) / (2.0 * dx)
            if n > 0:
                # method A: ghost values from the coarser level (with method C,
                # from its substituted field of the same face)
                lo_src = hat[(n - 1, ax, 1)] if coarse_side == "C" else phi[n - 1]
                hi_src = hat[(n - 1, ax, -1)] if coarse_side == "C" else phi[n - 1]
                minus_g = ghost_face(lo_src, N, ax, -1)
                plus_g = ghost_face(hi_src, N, ax, N)
                d[tuple(sl_lo)] = (plus[tuple(sl_lo)] - minus_g) / (2.0 * dx)
                d[tuple(sl_hi)] = (plus_g - minus[tuple(sl_hi)]) / (2.0 * dx)
            else:
                # outer boundary: one-sided, second order
                def at(i):
                    s = [slice(None)] * 3
                    s[ax] = slice(i, i + 1)
                    return p[tuple(s)]
                d[tuple(sl_lo)] = (-3.0 * at(0) + 4.0 * at(1) - at(2)) / (2.0 * dx)
                d[tuple(sl_hi)] = (3.0 * at(N - 1) - 4.0 * at(N - 2) + at(N - 3)) / (2.0 * dx)
            g[n, comp] = -d
    return g
