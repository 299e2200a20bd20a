"""Parity of the CUDA acceleration (g = -grad Phi: Eq. 8 stencil, Eqs. 3-6
ghost values on the fine side of each interface, children means on the coarse
side, Appendix A methods A and B) with the oracle, on the same potential.

The kernel and the oracle evaluate the same differences; they differ only in
the rounding of 1/(2 dx) and in the summation order of the 2^3 children, so
the bound is max|g_gpu - g_orc| <= 1e-12 max|g_orc| (observed ~1e-16)."""
import numpy as np
import pytest

import oracle
from paper_2301_06763_gb300 import workloads as wl
from tests.gpu_helpers import nm, rel_max

pytestmark = pytest.mark.gpu

ACCEL_REL_MAX = 1e-12


def gpu_accel(phi, N, dx0, precision="fp64", coarse_side="mean", iters=32):
    import torch
    m = nm()
    L = phi.shape[0]
    with m.Plan(L, N, dx0, 1.0, precision=precision) as plan:
        p = torch.from_numpy(np.ascontiguousarray(phi)).to("cuda", torch.float64)
        g = plan.acceleration(p, coarse_side=coarse_side, iters=iters)
        torch.cuda.synchronize()
        return g.cpu().numpy()


@pytest.mark.parametrize("L,N,seed", [(1, 4, 0), (2, 4, 1), (3, 8, 2), (4, 16, 3), (2, 32, 4), (5, 8, 5),
                                      (16, 4, 6), (3, 64, 7)])
def test_random_potential_matches_oracle(L, N, seed):
    # the stencil is defined for any field: an unstructured one exercises every
    # branch (interior, both interface sides, outer boundary) with no cancellation
    phi = np.random.default_rng(seed).standard_normal((L, N, N, N))
    dx0 = 1.0 / N
    g = gpu_accel(phi, N, dx0)
    ref = oracle.acceleration(phi, N, dx0)
    assert g.shape == ref.shape
    assert rel_max(g, ref) <= ACCEL_REL_MAX


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_acceleration_of_a_gpu_potential(precision):
    # the whole path: GPU potential, then GPU acceleration of it, against the
    # oracle's acceleration of the same GPU potential
    import torch
    m = nm()
    w = wl.config_binary()
    rho = w.rho()
    dt = torch.float32 if precision == "fp32" else torch.float64
    with m.Plan(w.levels, w.N, w.dx0, 1.0, precision=precision) as plan:
        phi = plan.potential(torch.from_numpy(rho).to("cuda", dt))
        g = plan.acceleration(phi)
        torch.cuda.synchronize()
        phi, g = phi.cpu().numpy(), g.cpu().numpy()
    assert rel_max(g, oracle.acceleration(phi, w.N, w.dx0)) <= ACCEL_REL_MAX


def test_full_size_6x128():
    # the benchmarked mesh size: every cell against the (vectorised) oracle
    N, L = 128, 6
    phi = np.random.default_rng(11).standard_normal((L, N, N, N))
    g = gpu_accel(phi, N, 1.0 / N)
    assert rel_max(g, oracle.acceleration(phi, N, 1.0 / N)) <= ACCEL_REL_MAX


def test_linear_potential_exact_on_gpu():
    # a closed form the stencil reproduces exactly at every cell of every
    # level, interfaces and outer boundary included
    N, L, dx0 = 16, 4, 0.3
    phi = np.empty((L, N, N, N))
    for k in range(L):
        c = wl.level_centres(N, dx0, k)
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        phi[k] = 1.5 * X - 0.25 * Y + 2.0 * Z - 3.0
    g = gpu_accel(phi, N, dx0)
    for comp, val in enumerate((-1.5, 0.25, -2.0)):
        assert np.allclose(g[:, comp], val, rtol=0, atol=1e-11)


def test_rejects_null_and_misshaped():
    import torch
    m = nm()
    with m.Plan(2, 8, 0.1, 1.0) as plan:
        phi = torch.zeros((2, 8, 8, 8), dtype=torch.float64, device="cuda")
        with pytest.raises(ValueError):
            plan.acceleration(phi, g=torch.zeros((2, 8, 8, 8), dtype=torch.float64, device="cuda"))
        with pytest.raises((TypeError, ValueError)):
            plan.acceleration(phi.float())


@pytest.mark.parametrize("L,N,seed,iters", [(2, 4, 20, 32), (3, 8, 21, 32), (4, 16, 22, 32), (2, 32, 23, 5),
                                            (3, 64, 24, 32), (5, 8, 25, 1), (2, 256, 26, 32)])
def test_method_C_matches_oracle(L, N, seed, iters):
    # Appendix A method C: face arrays swept `iters` times on the GPU (Jacobi
    # in the simplified form V = A - 1/8 sum of diagonal partners) against the
    # oracle's literal steps (ghosts by Eqs. 3-6, then the face condition)
    phi = np.random.default_rng(seed).standard_normal((L, N, N, N))
    dx0 = 1.0 / N
    g = gpu_accel(phi, N, dx0, coarse_side="flux", iters=iters)
    ref = oracle.acceleration(phi, N, dx0, coarse_side="C", iters=iters)
    assert rel_max(g, ref) <= ACCEL_REL_MAX


def test_method_C_full_size_6x128():
    N, L = 128, 6
    phi = np.random.default_rng(27).standard_normal((L, N, N, N))
    g = gpu_accel(phi, N, 1.0 / N, coarse_side="flux")
    assert rel_max(g, oracle.acceleration(phi, N, 1.0 / N, coarse_side="C")) <= ACCEL_REL_MAX
