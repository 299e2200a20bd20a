"""Failure detection without a GPU fault: the TMA-fed z-seam's mbarrier waits
are bounded; when they run out (a test hook stops the loads, so nothing ever
completes them) the kernel raises NM_ETIMEOUT in the device status word and
returns, and the context stays usable."""
import numpy as np
import pytest

import oracle
from paper_2301_06763_gb300 import workloads as wl
from tests.gpu_helpers import FP32_REL_MAX, nm, rel_max

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    import torch
    m = nm()
    L, N = 2, 16
    rho_np = wl.random_density(4, L, N)
    rho = torch.from_numpy(rho_np).to("cuda", torch.float32)
    with m.Plan(L, N, 1.0 / N, precision="fp32") as p:
        p.set_schedule(group=2, radix=16, tile=0, pipeline=1, fuse=0)
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


def test_status_is_clean_after_normal_solves():
    import torch
    m = nm()
    rho = torch.from_numpy(wl.random_density(5, 3, 32)).to("cuda", torch.float32)
    with m.Plan(3, 32, 1.0 / 32, precision="fp32") as p:
        for pipe in (0, 1):
            for fuse in (0, 1):
                p.set_schedule(group=3, radix=16, tile=0, pipeline=pipe, fuse=fuse)
                p.potential(rho)
    assert m.device_status(clear=True) == m.NM_OK
