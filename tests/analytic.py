"""Closed-form potentials used to pin the oracle (G = 1 unless given).

Each is written from the mathematics (shell theorem, or the classical closed
form for a uniform rectangular prism), independently of the oracle's code.
"""
import math

import numpy as np


def plummer(r, M, a, G=1.0):
    return -G * M / np.sqrt(r * r + a * a)


def uniform_sphere(r, M, R, G=1.0):
    r = np.asarray(r, dtype=float)
    inside = -G * M * (3.0 * R * R - r * r) / (2.0 * R ** 3)
    with np.errstate(divide="ignore"):
        outside = -G * M / np.where(r > 0, r, 1.0)
    return np.where(r <= R, inside, outside)


def poly_sphere(r, M, R, G=1.0):
    """rho = rho0 (1 - s^2)^2, s = r/R, inside R.  Shell theorem:
    Phi(r) = -G M(<r)/r - 4 pi G int_r^R rho(t) t dt."""
    r = np.asarray(r, dtype=float)
    rho0 = M / (4.0 * math.pi * R ** 3 * 8.0 / 105.0)
    s = np.clip(r / R, 0.0, 1.0)
    # M(<r) = 4 pi rho0 R^3 (s^3/3 - 2 s^5/5 + s^7/7)
    m_in = 4.0 * math.pi * rho0 * R ** 3 * (s ** 3 / 3.0 - 2.0 * s ** 5 / 5.0 + s ** 7 / 7.0)
    # int_r^R rho t dt = rho0 R^2 [F(1) - F(s)], F(s) = s^2/2 - s^4/2 + s^6/6
    F = lambda u: u ** 2 / 2.0 - u ** 4 / 2.0 + u ** 6 / 6.0
    outer = rho0 * R ** 2 * (F(1.0) - F(s))
    with np.errstate(divide="ignore", invalid="ignore"):
        phi_in = np.where(r > 0, -G * m_in / np.where(r > 0, r, 1.0), 0.0) \
            - 4.0 * math.pi * G * outer
    phi_out = -G * M / np.where(r > 0, r, 1.0)
    return np.where(r < R, phi_in, phi_out)


def box_integral(px, py, pz, x1, x2, y1, y2, z1, z2):
    """Integral of 1/|p - q| over q in the box [x1,x2]x[y1,y2]x[z1,z2].

    Classical closed form: sum over the 8 corners with sign (-1)^(i+j+k) of
      x y ln(z + R) + y z ln(x + R) + z x ln(y + R)
      - x^2/2 atan(y z / (x R)) - y^2/2 atan(z x / (y R)) - z^2/2 atan(x y / (z R)),
    (x, y, z) the corner relative to p and R its distance.  Terms whose
    coefficient vanishes are dropped (their limits are zero).
    """
    def F(x, y, z):
        R = math.sqrt(x * x + y * y + z * z)
        v = 0.0
        if x != 0 and y != 0:
            v += x * y * math.log(z + R)
        if y != 0 and z != 0:
            v += y * z * math.log(x + R)
        if z != 0 and x != 0:
            v += z * x * math.log(y + R)
        if x != 0:
            v -= 0.5 * x * x * math.atan(y * z / (x * R))
        if y != 0:
            v -= 0.5 * y * y * math.atan(z * x / (y * R))
        if z != 0:
            v -= 0.5 * z * z * math.atan(x * y / (z * R))
        return v

    tot = 0.0
    for i, X in enumerate((x1 - px, x2 - px)):
        for j, Y in enumerate((y1 - py, y2 - py)):
            for k, Z in enumerate((z1 - pz, z2 - pz)):
                s = 1.0 if (i + j + k) % 2 == 1 else -1.0
                tot += s * F(X, Y, Z)
    return tot


def oblate_spheroid(x, y, z, a, c, rho=1.0, G=1.0):
    """Homogeneous oblate spheroid x^2/a^2 + y^2/a^2 + z^2/c^2 <= 1 (a > c).

    Classical ellipsoid potential (Chandrasekhar 1969):
      Phi = -pi G rho a^2 c [J0 - (x^2 + y^2) J1 - z^2 J3],
      J0 = int_l^inf du / D(u),  J1 = int du / ((a^2+u) D),  J3 = int du / ((c^2+u) D),
      D(u) = (a^2 + u) sqrt(c^2 + u),
    with l = 0 inside and, outside, the positive root of
    (x^2 + y^2)/(a^2 + l) + z^2/(c^2 + l) = 1.  With s = sqrt(c^2 + u) and
    e2 = a^2 - c^2 the integrals are elementary (s0 = sqrt(c^2 + l)):
      J0 = 2/sqrt(e2) atan(sqrt(e2)/s0)
      J1 = atan(sqrt(e2)/s0)/e2^1.5 - s0/(e2 (e2 + s0^2))
      J3 = 2/(e2 s0) - 2 atan(sqrt(e2)/s0)/e2^1.5
    """
    x, y, z = (np.asarray(v, dtype=float) for v in (x, y, z))
    R2 = x * x + y * y
    z2 = z * z
    B = a * a + c * c - R2 - z2
    C = a * a * c * c - R2 * c * c - z2 * a * a
    disc = np.sqrt(np.maximum(B * B - 4.0 * C, 0.0))
    lam = np.where(R2 / (a * a) + z2 / (c * c) <= 1.0, 0.0, 0.5 * (-B + disc))
    e2 = a * a - c * c
    s0 = np.sqrt(c * c + lam)
    at = np.arctan(np.sqrt(e2) / s0)
    J0 = 2.0 / np.sqrt(e2) * at
    J1 = at / e2 ** 1.5 - s0 / (e2 * (e2 + s0 * s0))
    J3 = 2.0 / (e2 * s0) - 2.0 * at / e2 ** 1.5
    return -math.pi * G * rho * a * a * c * (J0 - R2 * J1 - z2 * J3)


def oblate_spheroid_accel(x, y, z, a, c, rho=1.0, G=1.0):
    """g = -grad Phi of `oblate_spheroid`: the derivative through the lower
    limit vanishes (the integrand is zero there), so
    g = -2 pi G rho a^2 c (x J1, y J1, z J3)."""
    x, y, z = (np.asarray(v, dtype=float) for v in (x, y, z))
    R2, z2 = x * x + y * y, z * z
    B = a * a + c * c - R2 - z2
    C = a * a * c * c - R2 * c * c - z2 * a * a
    disc = np.sqrt(np.maximum(B * B - 4.0 * C, 0.0))
    lam = np.where(R2 / (a * a) + z2 / (c * c) <= 1.0, 0.0, 0.5 * (-B + disc))
    e2 = a * a - c * c
    s0 = np.sqrt(c * c + lam)
    at = np.arctan(np.sqrt(e2) / s0)
    J1 = at / e2 ** 1.5 - s0 / (e2 * (e2 + s0 * s0))
    J3 = 2.0 / (e2 * s0) - 2.0 * at / e2 ** 1.5
    k = -2.0 * math.pi * G * rho * a * a * c
    return k * x * J1, k * y * J1, k * z * J3


def sphere_accel(dx, dy, dz, M, R, G=1.0):
    """Uniform sphere: g = -G M r_vec / R^3 inside, -G M r_vec / r^3 outside."""
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    f = np.where(r <= R, -G * M / R ** 3, -G * M / np.maximum(r, 1e-300) ** 3)
    return f * dx, f * dy, f * dz


def poly_sphere_accel_radial(r, M, R, G=1.0):
    """|g| of the C^1 polynomial sphere: G M(<r) / r^2."""
    r = np.asarray(r, dtype=float)
    rho0 = M / (4.0 * math.pi * R ** 3 * 8.0 / 105.0)
    s = np.clip(r / R, 0.0, 1.0)
    m_in = 4.0 * math.pi * rho0 * R ** 3 * (s ** 3 / 3.0 - 2.0 * s ** 5 / 5.0 + s ** 7 / 7.0)
    return G * m_in / np.maximum(r, 1e-300) ** 2


def box_integral_grid(px, py, pz, h):
    """`box_integral` over the cube [-h, h]^3 at every point of the arrays
    (px, py, pz): the same closed form, vectorised."""
    px, py, pz = (np.asarray(v, dtype=float) for v in (px, py, pz))

    def F(x, y, z):
        R = np.sqrt(x * x + y * y + z * z)
        v = np.zeros_like(R)
        with np.errstate(divide="ignore", invalid="ignore"):
            v += np.where((x != 0) & (y != 0), x * y * np.log(z + R), 0.0)
            v += np.where((y != 0) & (z != 0), y * z * np.log(x + R), 0.0)
            v += np.where((z != 0) & (x != 0), z * x * np.log(y + R), 0.0)
            v -= np.where(x != 0, 0.5 * x * x * np.arctan(y * z / (x * R)), 0.0)
            v -= np.where(y != 0, 0.5 * y * y * np.arctan(z * x / (y * R)), 0.0)
            v -= np.where(z != 0, 0.5 * z * z * np.arctan(x * y / (z * R)), 0.0)
        return v

    tot = np.zeros(np.broadcast(px, py, pz).shape)
    for i, X in enumerate((-h - px, h - px)):
        for j, Y in enumerate((-h - py, h - py)):
            for k, Z in enumerate((-h - pz, h - pz)):
                s = 1.0 if (i + j + k) % 2 == 1 else -1.0
                tot = tot + s * F(X, Y, Z)
    return tot


def workload_potential(workload, level):
    """The closed-form potential of a workload's density components at the
    cell centres of `level` (shape (N, N, N), [z, y, x]): Plummer spheres and
    homogeneous spheres by the shell theorem, a uniform background by the
    prism formula over the coarsest cube (side N dx0, where the nested mesh
    holds it).  Mass the mesh does not hold (a Plummer sphere's tail outside
    the coarsest cube) is included, so the difference to a mesh solution
    carries that truncation as well as the discretisation error."""
    w = workload
    N, dx = w.N, w.dx0 / 2.0 ** level
    c = -N * dx / 2.0 + (np.arange(N) + 0.5) * dx
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    out = np.zeros((N, N, N))
    for comp in w.components:
        kind = type(comp).__name__
        if kind in ("Plummer", "UniformSphere", "PolySphere"):
            cx, cy, cz = comp.centre
            r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2)
            if kind == "Plummer":
                out += plummer(r, comp.mass, comp.scale, w.G)
            elif kind == "UniformSphere":
                out += uniform_sphere(r, comp.mass, comp.radius, w.G)
            else:
                out += poly_sphere(r, comp.mass, comp.radius, w.G)
        elif kind == "Background":
            out += -w.G * comp.value * box_integral_grid(x, y, z, 0.5 * N * w.dx0)
        else:
            raise ValueError("no closed form for %s" % kind)
    return out
