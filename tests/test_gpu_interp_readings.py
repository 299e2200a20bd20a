"""Parity of both readings of the Fig. 6 interpolation with the oracle's, for
both methods and both precisions, through solo solves, batches and graph
replays: the carried Eqs. 3-6 rule (NM_INTERP_DIAGONAL, the default) and the
tensor-product trilinear one (NM_INTERP_TRILINEAR)."""
import numpy as np
import pytest

import oracle
from paper_2301_06763_gb300 import workloads as wl
from tests.gpu_helpers import (FP32_REL_L2, FP32_REL_MAX, FP64_REL_MAX, gpu_solve, nm, rel_l2,
                               rel_max)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,N,seed", [(1, 8, 0), (2, 4, 1), (2, 8, 2), (3, 8, 3), (4, 16, 4), (6, 8, 5),
                                      (3, 32, 6), (16, 4, 7)])
@pytest.mark.parametrize("method", ["original", "dipole"])
@pytest.mark.parametrize("interp", ["diagonal", "trilinear"])
def test_fp64_random_densities(L, N, seed, method, interp):
    rho = wl.random_density(seed, L, N, positive=False)
    dx0 = 0.41 / N
    ref = oracle.solve(rho, N, dx0, G=1.3, method=method, interp=interp)
    got = gpu_solve(rho, N, dx0, G=1.3, method=method, interp=interp)
    assert rel_max(got, ref) <= FP64_REL_MAX


@pytest.mark.parametrize("method", ["original", "dipole"])
@pytest.mark.parametrize("interp", ["diagonal", "trilinear"])
def test_fp32_binary_4x64(method, interp):
    w = wl.config_binary()
    rho = w.rho()
    ref = oracle.solve(rho, w.N, w.dx0, method=method, interp=interp)
    got = gpu_solve(rho.astype(np.float32), w.N, w.dx0, precision="fp32", method=method, interp=interp)
    assert rel_l2(got, ref) <= FP32_REL_L2
    assert rel_max(got, ref) <= FP32_REL_MAX


def test_differs_from_trilinear_where_it_should():
    # the two readings agree on the coarsest level and differ on finer ones
    rho = wl.random_density(9, 3, 16)
    a = gpu_solve(rho, 16, 1.0 / 16, interp="diagonal")
    b = gpu_solve(rho, 16, 1.0 / 16, interp="trilinear")
    assert np.array_equal(a[0], b[0])
    assert np.max(np.abs(a[2] - b[2])) > 1e-6 * np.max(np.abs(b[2]))


def test_batch_and_replay_equal_solo():
    import torch
    m = nm()
    shapes = [(4, 16), (3, 8), (5, 16), (2, 32)]
    plans, rhos, phis, solo = [], [], [], []
    try:
        for i, (L, N) in enumerate(shapes):
            p = m.Plan(L, N, 1.0 / N, interp="diagonal" if i % 2 == 0 else "trilinear")
            plans.append(p)
            r = torch.from_numpy(wl.random_density(30 + i, L, N)).cuda()
            rhos.append(r)
            phis.append(torch.empty((L, N, N, N), dtype=torch.float64, device="cuda"))
            solo.append(p.potential(r).clone())
        for _ in range(3):     # first call eager, then graph replays
            m.batch_potential(plans, rhos, phis)
            torch.cuda.synchronize()
            for s, f in zip(solo, phis):
                assert torch.equal(s, f)
    finally:
        for p in plans:
            p.close()

