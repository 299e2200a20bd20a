"""NM_FP64X: the transforms in double-float (two floats per value, ~48
significant bits) on the FP32 pipe, densities and potentials in double.
Against the FP64 oracle it must stay within 1e-12 of max|Phi| (the native
FP64 path's bound is 1e-11; double-float rounding is ~2^-46 per operation and
a transform of P = 2N points has log2 P stages)."""
import numpy as np
import pytest

import oracle
from paper_2301_06763_gb300 import workloads as wl
from tests.gpu_helpers import gpu_solve, nm, rel_max

pytestmark = pytest.mark.gpu

FP64X_REL_MAX = 1e-12


@pytest.mark.parametrize("L,N,seed", [(1, 8, 0), (2, 16, 1), (3, 8, 2), (4, 32, 3), (2, 64, 4), (6, 16, 5)])
@pytest.mark.parametrize("interp", ["diagonal", "trilinear"])
def test_matches_oracle(L, N, seed, interp):
    rho = wl.random_density(seed, L, N, positive=False)
    dx0 = 0.9 / N
    ref = oracle.solve(rho, N, dx0, G=1.2, interp=interp)
    got = gpu_solve(rho, N, dx0, G=1.2, precision="fp64x", interp=interp)
    assert rel_max(got, ref) <= FP64X_REL_MAX


def test_full_size_6x128_samples():
    # the benchmarked mesh size, every level, against the FP64 path on the GPU
    # (itself pinned to the oracle at 1e-11 in the full-size tests)
    w = wl.config_contrast(levels=6, N=128)
    rho = w.rho()
    a = gpu_solve(rho, w.N, w.dx0, precision="fp64x")
    b = gpu_solve(rho, w.N, w.dx0, precision="fp64")
    assert rel_max(a, b) <= FP64X_REL_MAX


def test_batch_with_other_precisions_equals_solo():
    import torch
    m = nm()
    shapes = [(3, 16, "fp64x"), (2, 32, "fp32"), (4, 16, "fp64"), (2, 64, "fp64x")]
    plans, rhos, phis, solo = [], [], [], []
    try:
        for i, (L, N, prec) in enumerate(shapes):
            p = m.Plan(L, N, 1.0 / N, precision=prec)
            plans.append(p)
            dt = torch.float32 if prec == "fp32" else torch.float64
            r = torch.from_numpy(wl.random_density(80 + i, L, N)).to("cuda", dt)
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


def test_unsupported_combinations():
    m = nm()
    for kw in ({"method": "dipole"}, {"method": "dipole3"}):
        with pytest.raises(m.NMError) as e:
            m.Plan(3, 16, 0.1, precision="fp64x", **kw)
        assert e.value.status == m.NM_EUNSUPPORTED
    with pytest.raises(m.NMError) as e:
        m.Plan(2, 4, 0.1, precision="fp64x")
    assert e.value.status == m.NM_EUNSUPPORTED
