"""CUDA path against the FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2301_06763_gb300 import workloads as wl
from tests.gpu_helpers import (FP32_REL_L2, FP32_REL_MAX, FP64_REL_MAX, gpu_solve, nm, rel_l2,
                               rel_max)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N", [4, 8, 16, 64])
def test_green_octant_matches_oracle_spectrum(N):
    m = nm()
    with m.Plan(2, N, 1.0) as p:
        got = p.green_octant()
    ref = oracle.green_spectrum(N).real[: N + 1, : N + 1, : N + 1]
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


CASES = [
    # (name, levels, N, density seed or workload)
    ("random L1 N4", 1, 4, 1),
    ("random L2 N4", 2, 4, 2),
    ("random L3 N8", 3, 8, 3),
    ("random L4 N16", 4, 16, 4),
    ("random L2 N32", 2, 32, 5),
    ("random L5 N8", 5, 8, 6),
]


@pytest.mark.parametrize("name,L,N,seed", CASES)
@pytest.mark.parametrize("method", ["original", "dipole"])
def test_fp64_random_densities(name, L, N, seed, method):
    rho = wl.random_density(seed, L, N, positive=False)
    dx0 = 0.37 / N
    ref = oracle.solve(rho, N, dx0, G=1.7, method=method)
    got = gpu_solve(rho, N, dx0, G=1.7, method=method)
    assert rel_max(got, ref) <= FP64_REL_MAX


@pytest.mark.parametrize("method", ["original", "dipole"])
def test_fp64_plummer_2x16(method):
    w = wl.config_small()
    rho = w.rho()
    ref = oracle.solve(rho, w.N, w.dx0, method=method)
    got = gpu_solve(rho, w.N, w.dx0, method=method)
    assert rel_max(got, ref) <= FP64_REL_MAX


@pytest.mark.parametrize("method", ["original", "dipole"])
def test_fp32_plummer_2x16(method):
    w = wl.config_small()
    rho = w.rho()
    ref = oracle.solve(rho, w.N, w.dx0, method=method)
    got = gpu_solve(rho.astype(np.float32), w.N, w.dx0, precision="fp32", method=method)
    assert rel_l2(got, ref) <= FP32_REL_L2
    assert rel_max(got, ref) <= FP32_REL_MAX


def test_fp64_and_fp32_binary_4x64():
    w = wl.config_binary()
    rho = w.rho()
    ref = oracle.solve(rho, w.N, w.dx0)
    got = gpu_solve(rho, w.N, w.dx0)
    assert rel_max(got, ref) <= FP64_REL_MAX
    got32 = gpu_solve(rho.astype(np.float32), w.N, w.dx0, precision="fp32")
    assert rel_l2(got32, ref) <= FP32_REL_L2
    assert rel_max(got32, ref) <= FP32_REL_MAX


def test_zero_density_gives_zero():
    got = gpu_solve(np.zeros((3, 16, 16, 16)), 16, 0.1)
    assert np.all(got == 0.0)


def test_point_mass_single_level_exact():
    N, dx = 32, 0.05
    rho = np.zeros((1, N, N, N))
    src = (3, 17, 30)
    rho[(0,) + src] = 2.0 / dx ** 3
    got = gpu_solve(rho, N, dx)[0]
    zz, yy, xx = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    r = dx * np.sqrt((zz - src[0]) ** 2 + (yy - src[1]) ** 2 + (xx - src[2]) ** 2)
    exp = -2.0 / np.where(r > 0, r, 1.0)
    exp[src] = -2.0 * oracle.SELF_TERM_C / dx
    assert rel_max(got, exp) <= FP64_REL_MAX
