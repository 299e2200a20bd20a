"""The three-level dipole scheme of Appendix B on the GPU: quadrupled grids
(Eqs. B.3-B.5, NM_METHOD_DIPOLE_TRIPLE) and their direct-sum replacement
(Eq. B.6, NM_METHOD_DIPOLE_TRIPLE_DIRECT) against the oracle, in both
precisions, solo and batched."""
import numpy as np
import pytest

import oracle
from paper_2301_06763_gb300 import workloads as wl
from tests.gpu_helpers import (FP32_REL_L2, FP32_REL_MAX, FP64_REL_MAX, gpu_solve, nm, rel_l2,
                               rel_max)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,N,seed", [(3, 4, 0), (3, 8, 1), (4, 8, 2), (5, 8, 3), (4, 16, 4), (3, 32, 5)])
@pytest.mark.parametrize("method", ["dipole3", "dipole3_ds"])
def test_fp64_matches_oracle(L, N, seed, method):
    rho = wl.random_density(seed, L, N, positive=False)
    dx0 = 0.7 / N
    ref = oracle.solve(rho, N, dx0, G=1.1, method=method)
    got = gpu_solve(rho, N, dx0, G=1.1, method=method)
    assert rel_max(got, ref) <= FP64_REL_MAX


@pytest.mark.parametrize("method", ["dipole3", "dipole3_ds"])
def test_fp32_matches_oracle(method):
    w = wl.config_binary()
    w = wl.Workload(w.name, 4, 32, w.dx0 * 2, w.components)
    rho = w.rho()
    ref = oracle.solve(rho, w.N, w.dx0, method=method)
    got = gpu_solve(rho.astype(np.float32), w.N, w.dx0, precision="fp32", method=method)
    assert rel_l2(got, ref) <= FP32_REL_L2
    assert rel_max(got, ref) <= FP32_REL_MAX


def test_keeps_a_dipole_two_levels_down():
    # the +-q pair of the oracle pin, on the GPU: nothing on level 0 with the
    # pairwise scheme, the point-dipole field with Eq. B.6
    N, L, dx0 = 16, 3, 1.0
    rho = np.zeros((L, N, N, N))
    rho[2, 8, 8, 8], rho[2, 8, 8, 9] = 1.0, -1.0
    two = gpu_solve(rho, N, dx0, method="dipole")
    ds = gpu_solve(rho, N, dx0, method="dipole3_ds")
    # (rounding noise only: two real fields share each complex transform)
    assert np.max(np.abs(two[0])) < 1e-12 * np.max(np.abs(ds[0]))
    g = oracle.Geometry(L, N, dx0)
    c0, c2 = g.centres(0), g.centres(2)
    Z, Y, X = np.meshgrid(c0, c0, c0, indexing="ij")
    m = g.dx(2) ** 3
    ref = -m / np.sqrt((X - c2[8]) ** 2 + (Y - c2[8]) ** 2 + (Z - c2[8]) ** 2) + \
        m / np.sqrt((X - c2[9]) ** 2 + (Y - c2[8]) ** 2 + (Z - c2[8]) ** 2)
    assert np.allclose(ds[0], ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_batch_and_replay_equal_solo():
    import torch
    m = nm()
    shapes = [(3, 16, "dipole3"), (4, 8, "dipole3_ds"), (5, 8, "dipole3"), (3, 8, "original")]
    plans, rhos, phis, solo = [], [], [], []
    try:
        for i, (L, N, meth) in enumerate(shapes):
            p = m.Plan(L, N, 1.0 / N, method=meth)
            plans.append(p)
            r = torch.from_numpy(wl.random_density(40 + i, L, N)).cuda()
            rhos.append(r)
            phis.append(torch.empty((L, N, N, N), dtype=torch.float64, device="cuda"))
            solo.append(p.potential(r).clone())
        for _ in range(3):
            m.batch_potential(plans, rhos, phis)
            torch.cuda.synchronize()
            for s, f in zip(solo, phis):
                assert torch.equal(s, f)
    finally:
        for p in plans:
            p.close()


def test_rejects_quadrupled_grid_beyond_1024_points():
    m = nm()
    with pytest.raises(m.NMError) as e:
        m.Plan(3, 256, 1.0, method="dipole3")
    assert e.value.status == m.NM_EUNSUPPORTED
