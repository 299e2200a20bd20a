"""The paired z-seam as a persistent pipeline (schedule pipeline = 3, 2N = 256):
the same transforms as the paired kernel (pipeline = 2), equal to it to FP32
rounding for every level-group size (one to all pairs per launch, with and
without the finest level's half-spectrum pair), bitwise equal between a batch
and solo solves, and checked against the FP64 oracle at sampled cells of the
full benchmark mesh."""
import numpy as np
import pytest

import oracle
from paper_2301_06763_gb300 import workloads as wl
from tests.gpu_helpers import FP32_REL_L2, FP32_REL_MAX, nm, rel_l2, rel_max

pytestmark = pytest.mark.gpu


def solve(rho, N, dx0, sched):
    import torch
    m = nm()
    L = rho.shape[0]
    with m.Plan(L, N, dx0, precision="fp32") as p:
        p.set_schedule(*sched)
        assert p.schedule()["pipeline"] == sched[3]
        r = torch.from_numpy(np.ascontiguousarray(rho, dtype=np.float32)).to("cuda")
        phi = p.potential(r)
        torch.cuda.synchronize()
        return phi.cpu().numpy()


@pytest.mark.parametrize("L,group", [(2, 2), (3, 1), (3, 2), (6, 6), (6, 4)])
def test_persistent_zseam_equals_paired_to_rounding(L, group):
    N = 128
    rho = wl.random_density(40 + L + group, L, N)
    a = solve(rho, N, 1.0 / N, (group, 16, 0, 2, 0))
    b = solve(rho, N, 1.0 / N, (group, 16, 0, 3, 0))
    assert rel_l2(b, a) <= 2e-7
    assert rel_max(b, a) <= 1e-6


def test_persistent_zseam_full_size_against_the_oracle():
    # the benchmark mesh; the oracle at interface and interior cells of every level
    w = wl.config_contrast()
    rho = w.rho()
    got = solve(rho, w.N, w.dx0, (w.levels, 16, 0, 3, 0))
    rng = np.random.default_rng(3)
    N = w.N
    cells = []
    for lev in range(w.levels):
        for (z, y, x) in [(0, 0, 0), (N // 4, N // 4, N // 4), (N // 4 - 1, N // 2, 3 * N // 4),
                          (N - 1, N - 1, N - 1)]:
            cells.append((lev, z, y, x))
        for _ in range(2):
            cells.append((lev,) + tuple(int(v) for v in rng.integers(0, N, 3)))
    ref = oracle.nested_potential_at(rho, N, w.dx0, cells)
    val = np.array([got[c] for c in cells])
    scale = np.abs(got).max()
    assert np.abs(val - ref).max() <= FP32_REL_MAX * scale
    assert rel_l2(val, ref) <= FP32_REL_L2 * 10


def test_persistent_zseam_in_a_batch_equals_solo():
    import torch
    m = nm()
    shapes = [(3, 128), (2, 128), (4, 64)]
    plans, rhos, phis, solo = [], [], [], []
    for i, (L, N) in enumerate(shapes):
        p = m.Plan(L, N, 0.9 / N, precision="fp32")
        if N == 128:
            p.set_schedule(L, 16, 0, 3, 0)
        r = torch.from_numpy(wl.random_density(60 + i, L, N)).to("cuda", torch.float32)
        plans.append(p)
        rhos.append(r)
        phis.append(torch.empty((L, N, N, N), dtype=torch.float64, device="cuda"))
        solo.append(p.potential(r).cpu().numpy())
    m.batch_potential(plans, rhos, phis)
    torch.cuda.synchronize()
    for f, s in zip(phis, solo):
        assert np.array_equal(f.cpu().numpy(), s)
    for p in plans:
        p.close()


def test_persistent_zseam_schedule_limits():
    m = nm()
    with m.Plan(2, 64, 1.0 / 64, precision="fp32") as p:       # 2N = 128: not this kernel's size
        with pytest.raises(m.NMError):
            p.set_schedule(2, 16, 0, 3, 0)
    with m.Plan(2, 128, 1.0 / 128, precision="fp32") as p:
        with pytest.raises(m.NMError):
            p.set_schedule(2, 16, 1, 3, 0)                       # narrow tiles only
        with pytest.raises(m.NMError):
            p.set_schedule(2, 8, 0, 3, 0)                        # 16 values per thread only
        with pytest.raises(m.NMError):
            p.set_schedule(2, 16, 0, 3, 1)                       # not fused
    with m.Plan(2, 128, 1.0 / 128, precision="fp64") as p:      # FP32 only
        with pytest.raises(m.NMError):
            p.set_schedule(2, 16, 0, 3, 0)
