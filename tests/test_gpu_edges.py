"""Edge cases of the CUDA path against the oracle: the most levels, the
smallest N, both methods and precisions mixed in one batch, and the doubled
grids at the largest N (transforms of 1024^3)."""
import numpy as np
import pytest

import oracle
from paper_2301_06763_gb300 import workloads as wl
from tests.gpu_helpers import FP32_REL_MAX, FP64_REL_MAX, gpu_solve, nm, rel_max

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method", ["original", "dipole"])
def test_sixteen_levels(method):
    L, N = 16, 8
    rho = wl.random_density(16, L, N)
    ref = oracle.solve(rho, N, 1.0 / N, method=method)
    assert rel_max(gpu_solve(rho, N, 1.0 / N, method=method), ref) <= FP64_REL_MAX
    got32 = gpu_solve(rho.astype(np.float32), N, 1.0 / N, precision="fp32", method=method)
    assert rel_max(got32, ref) <= FP32_REL_MAX


@pytest.mark.parametrize("method", ["original", "dipole"])
def test_smallest_mesh_many_levels(method):
    L, N = 10, 4
    rho = wl.random_density(4, L, N, positive=False)
    ref = oracle.solve(rho, N, 0.3, G=0.7, method=method)
    assert rel_max(gpu_solve(rho, N, 0.3, G=0.7, method=method), ref) <= FP64_REL_MAX


def test_mixed_batch_of_methods_and_precisions():
    import torch
    m = nm()
    spec = [(3, 16, "fp64", "dipole"), (2, 32, "fp32", "original"), (4, 8, "fp32", "dipole"),
            (2, 16, "fp64", "original"), (5, 4, "fp64", "dipole")]
    plans, rhos, phis, refs = [], [], [], []
    for i, (L, N, prec, meth) in enumerate(spec):
        rho = wl.random_density(50 + i, L, N)
        dt = torch.float32 if prec == "fp32" else torch.float64
        plans.append(m.Plan(L, N, 1.0 / N, precision=prec, method=meth))
        rhos.append(torch.from_numpy(rho).to("cuda", dt))
        phis.append(torch.empty((L, N, N, N), dtype=torch.float64, device="cuda"))
        refs.append(oracle.solve(rho, N, 1.0 / N, method=meth))
    solo = [p.potential(r).cpu().numpy() for p, r in zip(plans, rhos)]
    for _ in range(3):
        m.batch_potential(plans, rhos, phis)
    torch.cuda.synchronize()
    for (L, N, prec, meth), f, s, ref in zip(spec, phis, solo, refs):
        got = f.cpu().numpy()
        assert np.array_equal(got, s)
        assert rel_max(got, ref) <= (FP64_REL_MAX if prec == "fp64" else FP32_REL_MAX)
    for p in plans:
        p.close()


def test_dipole_at_the_largest_mesh():
    # N = 256: the doubled fine grid is 512^3 cells in a 1024^3 transform
    w = wl.Workload("poly-2x256", 2, 256, 1.0 / 256, [wl.PolySphere(1.0, 0.1, (0.01, 0.0, -0.02))])
    rho = w.rho()
    got = gpu_solve(rho.astype(np.float32), w.N, w.dx0, precision="fp32", method="dipole")
    sm = [(0, 128, 128, 128), (0, 3, 250, 77), (0, 64, 100, 191), (1, 128, 128, 128)]
    ref = oracle.nested_potential_at(rho, w.N, w.dx0, sm, method="dipole")
    vals = np.array([got[s] for s in sm])
    assert np.max(np.abs(vals - ref)) <= FP32_REL_MAX * np.max(np.abs(got))
