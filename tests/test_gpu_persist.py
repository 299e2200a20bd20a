"""The persistent schedule (fuse = 3): every step of the solves of a batch --
restriction, the five transform passes of every level pair, the carried
interpolation and the assembly of every mesh -- as work items of one launch
that CTAs take from a device ticket in dependency order.  Against the FP64
oracle, bitwise against solo solves in batches of uneven meshes (eager,
captured and replayed), with work slots reused within a mesh, and with its
bounded waits made to run out through the fault hook (no GPU fault)."""
import numpy as np
import pytest

import oracle
from paper_2301_06763_gb300 import workloads as wl
from tests.gpu_helpers import FP32_REL_L2, FP32_REL_MAX, nm, rel_l2, rel_max

pytestmark = pytest.mark.gpu


def persistent_plan(m, L, N, group=None, interp="diagonal"):
    p = m.Plan(L, N, 1.0 / N, precision="fp32", interp=interp)
    p.set_schedule(group or L, 16, 0, 0, 3)
    assert p.schedule()["fuse"] == 3
    return p


@pytest.mark.parametrize("L,N,group,interp", [(1, 32, None, "diagonal"), (2, 32, None, "trilinear"),
                                              (5, 32, 2, "diagonal"), (4, 64, None, "diagonal"),
                                              (3, 64, 1, "trilinear"), (2, 128, None, "diagonal")])
def test_persistent_solve_matches_the_oracle(L, N, group, interp):
    import torch
    m = nm()
    rho = wl.random_density(60 + L + N, L, N)
    ref = oracle.solve(rho, N, 1.0 / N, interp=interp)
    with persistent_plan(m, L, N, group, interp) as p:
        got = p.potential(torch.from_numpy(rho).to("cuda", torch.float32)).cpu().numpy()
    assert rel_l2(got, ref) <= FP32_REL_L2 and rel_max(got, ref) <= FP32_REL_MAX


def test_persistent_256_cubed_sampled():
    import torch
    m = nm()
    w = wl.Workload("poly-3x256", 3, 256, 1.0 / 256, [wl.PolySphere(1.0, 0.2)])
    rho = w.rho()
    cells = [(0, 128, 128, 128), (1, 63, 64, 192), (2, 255, 0, 128)]
    ref = oracle.nested_potential_at(rho, w.N, w.dx0, cells)
    with persistent_plan(m, 3, 256) as p:
        got = p.potential(torch.from_numpy(rho).to("cuda", torch.float32)).cpu().numpy()
    vals = np.array([got[c] for c in cells])
    assert np.max(np.abs(vals - ref)) <= FP32_REL_MAX * np.max(np.abs(got))


def test_batch_of_uneven_meshes_is_one_launch_and_equals_solo():
    import torch
    m = nm()
    meshes = wl.config_batch(seed=2, count=12)
    plans, rhos, phis, solo = [], [], [], []
    for i, w in enumerate(meshes):
        p = persistent_plan(m, w.levels, w.N, group=max(1, w.levels // 2) if i % 3 == 0 else None)
        r = torch.from_numpy(w.rho()).to("cuda", torch.float32)
        plans.append(p)
        rhos.append(r)
        phis.append(torch.empty(r.shape, dtype=torch.float64, device="cuda"))
        solo.append(p.potential(r).cpu().numpy())
    for rep in range(3):      # eager, captured, replayed
        l0 = m.kernel_launches()
        m.batch_potential(plans, rhos, phis)
        torch.cuda.synchronize()
        assert m.kernel_launches() - l0 == 1
        for f, s in zip(phis, solo):
            assert np.array_equal(f.cpu().numpy(), s)
    assert m.device_status(clear=True) == m.NM_OK
    for p in plans:
        p.close()


def test_mixed_batch_persistent_and_round_based():
    import torch
    m = nm()
    shapes = [(3, 32, 3), (2, 64, 0), (4, 64, 3), (3, 128, 0), (2, 32, 3)]
    plans, rhos, phis, solo = [], [], [], []
    for i, (L, N, fuse) in enumerate(shapes):
        p = m.Plan(L, N, 1.0 / N, precision="fp32")
        if fuse == 3:
            p.set_schedule(L, 16, 0, 0, 3)
        r = torch.from_numpy(wl.random_density(70 + i, L, N)).to("cuda", torch.float32)
        plans.append(p)
        rhos.append(r)
        phis.append(torch.empty(r.shape, dtype=torch.float64, device="cuda"))
        solo.append(p.potential(r).cpu().numpy())
    for _ in range(2):
        m.batch_potential(plans, rhos, phis)
        torch.cuda.synchronize()
        for f, s in zip(phis, solo):
            assert np.array_equal(f.cpu().numpy(), s)
    for p in plans:
        p.close()


def test_bounded_waits_report_timeout_and_context_survives():
    # with the hook on, finished items go uncounted, so every dependent wait
    # runs out (0.1 s limit): the launch stops, NM_ETIMEOUT is in the status
    # word, and the next solve is correct
    import torch
    m = nm()
    L, N = 3, 32
    rho_np = wl.random_density(8, L, N)
    rho = torch.from_numpy(rho_np).to("cuda", torch.float32)
    with persistent_plan(m, L, N) as p:
        assert m.device_status(clear=True) == m.NM_OK
        m.debug_fault_timeout(True)
        try:
            p.potential(rho)
            st = m.device_status(clear=True)
        finally:
            m.debug_fault_timeout(False)
        assert st == m.NM_ETIMEOUT
        phi = p.potential(rho).cpu().numpy()
        assert m.device_status(clear=True) == m.NM_OK
    assert rel_max(phi, oracle.solve(rho_np, N, 1.0 / N)) <= FP32_REL_MAX


def test_persistent_schedule_validation():
    m = nm()
    with m.Plan(3, 32, 1.0 / 32, precision="fp32") as p:
        for bad in (dict(group=3, radix=16, tile=1, pipeline=0, fuse=3),
                    dict(group=3, radix=16, tile=0, pipeline=2, fuse=3),
                    dict(group=3, radix=8, tile=0, pipeline=0, fuse=3)):
            with pytest.raises(m.NMError):
                p.set_schedule(**bad)
    for kw in (dict(precision="fp64"), dict(precision="fp32", method="dipole")):
        with m.Plan(3, 32, 1.0 / 32, **kw) as p:
            with pytest.raises(m.NMError):
                p.set_schedule(3, 16, 0, 0, 3)
    with m.Plan(3, 16, 1.0 / 16, precision="fp32") as p:      # 2N >= 64
        with pytest.raises(m.NMError):
            p.set_schedule(3, 16, 0, 0, 3)
