"""Seeded synthetic densities for the nested-mesh potential solver.

This module only *generates inputs*: it samples analytic densities at the cell
centres of a nested mesh (levels centred on the origin, level m of cell size
dx0 / 2^m and N cells per axis, arrays indexed [level, z, y, x]).  It contains
none of the solver's arithmetic, so the CUDA path, the CPU oracle, the tests and
the benchmark can all draw the same inputs from it.

Densities follow the paper's test problems in spirit (compact, centrally
concentrated, analytic potentials known): Plummer spheres, homogeneous spheres
and a C^1 polynomial sphere.  All domains have base side 1.0 and G = 1.
"""
from dataclasses import dataclass, field
import math

import numpy as np


def level_centres(N, dx0, m):
    dx = dx0 / (2.0 ** m)
    return -N * dx / 2.0 + (np.arange(N) + 0.5) * dx


def sample(levels, N, dx0, density):
    """rho[m, z, y, x] = density(x, y, z) at every cell centre of every level."""
    out = np.empty((levels, N, N, N), dtype=np.float64)
    for m in range(levels):
        c = level_centres(N, dx0, m)
        z = c[:, None, None]
        y = c[None, :, None]
        x = c[None, None, :]
        out[m] = density(x, y, z)
    return out


# --- analytic density components ------------------------------------------------

@dataclass(frozen=True)
class Plummer:
    mass: float
    scale: float
    centre: tuple = (0.0, 0.0, 0.0)

    def density(self, x, y, z):
        cx, cy, cz = self.centre
        r2 = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2
        a = self.scale
        return 3.0 * self.mass / (4.0 * math.pi * a ** 3) * (1.0 + r2 / a ** 2) ** -2.5


@dataclass(frozen=True)
class UniformSphere:
    mass: float
    radius: float
    centre: tuple = (0.0, 0.0, 0.0)

    def density(self, x, y, z):
        cx, cy, cz = self.centre
        r2 = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2
        rho0 = 3.0 * self.mass / (4.0 * math.pi * self.radius ** 3)
        return np.where(r2 <= self.radius ** 2, rho0, 0.0)


@dataclass(frozen=True)
class PolySphere:
    """rho = rho0 (1 - r^2/R^2)^2 inside R (C^1 at the surface)."""
    mass: float
    radius: float
    centre: tuple = (0.0, 0.0, 0.0)

    def density(self, x, y, z):
        cx, cy, cz = self.centre
        R = self.radius
        r2 = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2
        rho0 = self.mass / (4.0 * math.pi * R ** 3 * 8.0 / 105.0)
        s = 1.0 - r2 / R ** 2
        return np.where(s > 0, rho0 * s * s, 0.0)


@dataclass(frozen=True)
class Background:
    value: float

    def density(self, x, y, z):
        return np.full(np.broadcast(x, y, z).shape, self.value)


@dataclass
class Workload:
    name: str
    levels: int
    N: int
    dx0: float
    components: list = field(default_factory=list)
    G: float = 1.0

    def density(self, x, y, z):
        tot = 0.0
        for c in self.components:
            tot = tot + c.density(x, y, z)
        return tot

    def rho(self):
        return sample(self.levels, self.N, self.dx0, self.density)


# --- the five configurations ------------------------------------------------------

def config_small():
    """2 levels of 16^3, one centred Plummer sphere (mass 1, scale 0.05)."""
    return Workload("plummer-2x16", 2, 16, 1.0 / 16, [Plummer(1.0, 0.05)])


def config_binary():
    """4 levels of 64^3: Plummer spheres of mass 1 and 0.5 (scale 0.02) at
    x = -0.03 and +0.03, plus a uniform background of 1e-4."""
    return Workload("binary-4x64", 4, 64, 1.0 / 64, [
        Plummer(1.0, 0.02, (-0.03, 0.0, 0.0)),
        Plummer(0.5, 0.02, (+0.03, 0.0, 0.0)),
        Background(1e-4),
    ])


def config_contrast(seed=0, levels=6, N=128):
    """levels x N^3: homogeneous sphere (radius 0.3, mass 1) plus a Plummer core
    (scale 1e-3, mass 0.037), central density contrast ~1e6; each centre is
    offset by U(-1/2, 1/2) finest-cell sizes per axis from a seeded generator."""
    rng = np.random.default_rng(seed)
    dx0 = 1.0 / N
    dxf = dx0 / 2.0 ** (levels - 1)
    c1 = tuple(float(v) for v in rng.uniform(-0.5, 0.5, 3) * dxf)
    c2 = tuple(float(v) for v in rng.uniform(-0.5, 0.5, 3) * dxf)
    return Workload("contrast-%dx%d" % (levels, N), levels, N, dx0, [
        UniformSphere(1.0, 0.3, c1), Plummer(0.037, 1e-3, c2)])


def random_plummers(rng, levels, N):
    """1-4 Plummer spheres: masses U(0.1, 1), scales log-U(1e-3, 1e-1), centres
    uniform inside the central half of the finest level."""
    dx0 = 1.0 / N
    half_finest = 0.5 * N * dx0 / 2.0 ** (levels - 1)
    comps = []
    for _ in range(int(rng.integers(1, 5))):
        mass = float(rng.uniform(0.1, 1.0))
        scale = float(math.exp(rng.uniform(math.log(1e-3), math.log(1e-1))))
        centre = tuple(float(v) for v in rng.uniform(-0.5, 0.5, 3) * half_finest)
        comps.append(Plummer(mass, scale, centre))
    return comps


def config_batch(seed=0, count=64, Ns=(32, 64, 128), level_range=(2, 8)):
    """``count`` independent meshes, N uniform over ``Ns``, levels uniform over
    ``level_range`` (inclusive), densities from ``random_plummers``."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(rng.choice(Ns))
        L = int(rng.integers(level_range[0], level_range[1] + 1))
        out.append(Workload("batch-%d" % i, L, N, 1.0 / N, random_plummers(rng, L, N)))
    return out


def config_serving(rate, count=2000, seed=0, Ns=(32, 64, 128, 256), level_range=(3, 10)):
    """Poisson arrivals at ``rate`` requests/s: list of (arrival_time_s, Workload)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        N = int(rng.choice(Ns))
        L = int(rng.integers(level_range[0], level_range[1] + 1))
        out.append((t, Workload("req-%d" % i, L, N, 1.0 / N, random_plummers(rng, L, N))))
    return out


def random_density(seed, levels, N, positive=True):
    """Unstructured seeded density (uniform random per cell) for parity tests."""
    rng = np.random.default_rng(seed)
    r = rng.random((levels, N, N, N))
    return r if positive else r - 0.5


# --- the paper's comparison problems (Sect. 2 and Sect. 5) ------------------------

@dataclass(frozen=True)
class HomogeneousSpheroid:
    """Uniform density inside x^2/a^2 + y^2/a^2 + z^2/c^2 <= 1."""
    a: float
    c: float
    rho: float = 1.0

    def density(self, x, y, z):
        inside = (x * x + y * y) / self.a ** 2 + z * z / self.c ** 2 <= 1.0
        return np.where(inside, self.rho, 0.0)


@dataclass(frozen=True)
class HomogeneousSphere:
    radius: float
    rho: float
    centre: tuple = (0.0, 0.0, 0.0)

    def density(self, x, y, z):
        cx, cy, cz = self.centre
        r2 = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2
        return np.where(r2 <= self.radius ** 2, self.rho, 0.0)


def config_paper_ellipsoid(N=128, levels=4):
    """Oblate homogeneous ellipsoid with semi-axes 1 : 1 : 0.5 (short axis on z)
    in the domain [-2.25, 2.25]^3, the paper's first test problem."""
    return Workload("ellipsoid-%dx%d" % (levels, N), levels, N, 4.5 / N, [HomogeneousSpheroid(1.0, 0.5)])


def config_paper_binary(N=128, levels=4):
    """Two homogeneous spheres of radius 0.2 centred at x = -0.5 and x = +0.5,
    the left one twice as massive, in [-2.25, 2.25]^3: the paper's binary star."""
    return Workload("binary-star-%dx%d" % (levels, N), levels, N, 4.5 / N, [
        HomogeneousSphere(0.2, 2.0, (-0.5, 0.0, 0.0)), HomogeneousSphere(0.2, 1.0, (0.5, 0.0, 0.0))])
