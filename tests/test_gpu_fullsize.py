"""The benchmark workload at full size (6 levels of 128^3): sampled cells
against the oracle's direct-summation route, and linearity."""
import numpy as np
import pytest

import oracle
from paper_2301_06763_gb300 import workloads as wl
from tests.gpu_helpers import FP32_REL_MAX, FP64_REL_MAX, gpu_solve, nm

pytestmark = pytest.mark.gpu


def samples(L, N, per_level=3, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for n in range(L):
        out.append((n, N // 2, N // 2, N // 2))               # centre
        out.append((n, 0, N - 1, N // 3))                     # level boundary
        out.append((n, N // 4 - 1, N // 4, 3 * N // 4))      # interface of the next level
        for _ in range(per_level):
            out.append((n, *map(int, rng.integers(0, N, 3))))
    return out


@pytest.fixture(scope="module")
def contrast():
    w = wl.config_contrast()
    rho = w.rho()
    sm = samples(w.levels, w.N)
    ref = oracle.nested_potential_at(rho, w.N, w.dx0, sm)
    return w, rho, sm, ref


def test_fp64_full_size_sampled(contrast):
    w, rho, sm, ref = contrast
    got = gpu_solve(rho, w.N, w.dx0)
    scale = np.max(np.abs(got))
    vals = np.array([got[s] for s in sm])
    assert np.max(np.abs(vals - ref)) <= FP64_REL_MAX * scale


def test_fp32_full_size_sampled(contrast):
    w, rho, sm, ref = contrast
    got = gpu_solve(rho.astype(np.float32), w.N, w.dx0, precision="fp32")
    scale = np.max(np.abs(got))
    vals = np.array([got[s] for s in sm])
    assert np.max(np.abs(vals - ref)) <= FP32_REL_MAX * scale


def test_linearity_full_size():
    w = wl.config_contrast()
    r1 = w.rho()
    r2 = wl.random_density(5, w.levels, w.N)
    a = gpu_solve(r1 + 2.0 * r2, w.N, w.dx0)
    b = gpu_solve(r1, w.N, w.dx0) + 2.0 * gpu_solve(r2, w.N, w.dx0)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


def test_dipole_binary_4x64_against_oracle():
    w = wl.config_binary()
    rho = w.rho()
    ref = oracle.solve(rho, w.N, w.dx0, method="dipole")
    got = gpu_solve(rho, w.N, w.dx0, method="dipole")
    assert np.max(np.abs(got - ref)) <= FP64_REL_MAX * np.max(np.abs(ref))
    got32 = gpu_solve(rho.astype(np.float32), w.N, w.dx0, precision="fp32", method="dipole")
    assert np.max(np.abs(got32 - ref)) <= FP32_REL_MAX * np.max(np.abs(ref))


def test_maximum_size_runs():
    # the largest built mesh: N = 256 (transforms of 512^3), 3 levels, FP32,
    # checked at sampled cells against direct sums
    w = wl.Workload("poly-3x256", 3, 256, 1.0 / 256, [wl.PolySphere(1.0, 0.2)])
    rho = w.rho()
    sm = [(0, 128, 128, 128), (1, 10, 200, 64), (2, 255, 0, 128)]
    ref = oracle.nested_potential_at(rho, w.N, w.dx0, sm)
    got = gpu_solve(rho.astype(np.float32), w.N, w.dx0, precision="fp32")
    vals = np.array([got[s] for s in sm])
    assert np.max(np.abs(vals - ref)) <= FP32_REL_MAX * np.max(np.abs(got))
