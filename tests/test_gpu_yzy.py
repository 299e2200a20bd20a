"""The three-pass form of the level convolutions (schedule fuse = 2): x-forward
into kx-major planes, one fused y/z/y pass per kx plane with its ky residues
split over a thread-block cluster, x-inverse.  Against the FP64 oracle on every
cell where it is affordable, at sampled cells by direct sums at 256^3, against
the five-pass form, for both cluster splits, one level (a full field alone)
and batches."""
import numpy as np
import pytest

import oracle
from paper_2301_06763_gb300 import workloads as wl
from tests.gpu_helpers import FP32_REL_L2, FP32_REL_MAX, nm, rel_l2, rel_max

pytestmark = pytest.mark.gpu

THREE_PASS = dict(group=16, radix=16, pipeline=0, fuse=2)


def solve(m, L, N, rho, sched=None, split=0):
    import torch
    with m.Plan(L, N, 1.0 / N, precision="fp32") as p:
        if sched == "three":
            p.set_schedule(min(16, L), 16, split, 0, 2)
            assert p.schedule()["fuse"] == 2
        elif sched is not None:
            p.set_schedule(**sched)
        out = p.potential(torch.from_numpy(rho).to("cuda", torch.float32)).cpu().numpy()
    return out


@pytest.mark.parametrize("L,N,split", [(1, 32, 0), (3, 32, 0), (4, 32, 0), (2, 64, 0), (3, 64, 1),
                                       (2, 128, 0), (2, 128, 1)])
def test_three_pass_against_the_oracle_every_cell(L, N, split):
    m = nm()
    rho = wl.random_density(40 + L + N + split, L, N)
    ref = oracle.solve(rho, N, 1.0 / N)
    got = solve(m, L, N, rho, "three", split)
    assert rel_l2(got, ref) <= FP32_REL_L2 and rel_max(got, ref) <= FP32_REL_MAX, (rel_l2(got, ref), rel_max(got, ref))


@pytest.mark.parametrize("L,N,split", [(6, 128, 0), (6, 128, 1), (5, 64, 0), (3, 256, 0)])
def test_three_pass_against_the_five_pass_form(L, N, split):
    # same mesh, same FP32 pipeline precision: the two forms differ only in
    # rounding order
    m = nm()
    rho = wl.config_contrast(levels=L, N=N).rho()
    a = solve(m, L, N, rho, "three", split)
    b = solve(m, L, N, rho, dict(group=L, radix=16, tile=0, pipeline=0, fuse=0))
    assert rel_l2(a, b) <= 1e-6 and rel_max(a, b) <= 5e-6


def test_three_pass_at_256_cubed_against_direct_sums():
    m = nm()
    L, N = 3, 256
    w = wl.Workload("poly-3x256", L, N, 1.0 / N, [wl.PolySphere(1.0, 0.2)])
    rho = w.rho()
    cells = [(0, 128, 128, 128), (1, 63, 64, 192), (2, 255, 0, 128), (2, 17, 250, 3)]
    ref = oracle.nested_potential_at(rho, N, w.dx0, cells)
    got = solve(m, L, N, rho, "three")
    vals = np.array([got[c] for c in cells])
    assert np.max(np.abs(vals - ref)) <= FP32_REL_MAX * np.max(np.abs(got))


def test_three_pass_batches_equal_solo_solves():
    import torch
    m = nm()
    shapes = [(3, 32), (2, 64), (4, 128), (2, 32), (3, 128)]
    plans, rhos, phis, solo = [], [], [], []
    for i, (L, N) in enumerate(shapes):
        rho = wl.random_density(90 + i, L, N)
        p = m.Plan(L, N, 1.0 / N, precision="fp32")
        p.set_schedule(L, 16, 0, 0, 2)
        plans.append(p)
        rhos.append(torch.from_numpy(rho).to("cuda", torch.float32))
        phis.append(torch.empty((L, N, N, N), dtype=torch.float64, device="cuda"))
        solo.append(p.potential(rhos[-1]).cpu().numpy())
    for _ in range(3):      # eager, captured, replayed
        m.batch_potential(plans, rhos, phis)
        torch.cuda.synchronize()
        for f, s in zip(phis, solo):
            assert np.array_equal(f.cpu().numpy(), s)
    for p in plans:
        p.close()


def test_three_pass_schedule_validation():
    m = nm()
    with m.Plan(3, 64, 1.0 / 64, precision="fp32") as p:
        for bad in (dict(group=1, radix=8, tile=0, pipeline=0, fuse=2),    # radix 16 only
                    dict(group=1, radix=16, tile=0, pipeline=2, fuse=2)):  # no z-seam choice
            with pytest.raises(m.NMError):
                p.set_schedule(**bad)
    with m.Plan(3, 64, 1.0 / 64, precision="fp64") as p:                   # FP32 only
        with pytest.raises(m.NMError):
            p.set_schedule(1, 16, 0, 0, 2)
    with m.Plan(3, 16, 1.0 / 16, precision="fp32") as p:                   # 2N >= 64
        with pytest.raises(m.NMError):
            p.set_schedule(1, 16, 0, 0, 2)
    with m.Plan(3, 32, 1.0 / 32, precision="fp32", method="dipole") as p:  # original method
        with pytest.raises(m.NMError):
            p.set_schedule(1, 16, 0, 0, 2)
