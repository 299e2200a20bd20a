"""Plan lifecycle: device memory comes back when plans are destroyed, and a
failed workspace allocation (host-side fault injection) returns NM_ENOMEM,
frees what it had allocated and leaves the library usable."""
import numpy as np
import pytest

from paper_2301_06763_gb300 import workloads as wl
from tests.gpu_helpers import nm

pytestmark = pytest.mark.gpu

KINDS = [dict(precision="fp32"), dict(precision="fp64"), dict(precision="fp64x"),
         dict(precision="fp32", method="dipole"), dict(precision="fp32", method="dipole3"),
         dict(precision="fp64", interp="trilinear")]


def churn(m, torch, rounds=3):
    for _ in range(rounds):
        for kw in KINDS:
            with m.Plan(4, 32, 1.0 / 32, **kw) as p:
                dt = torch.float32 if kw["precision"] == "fp32" else torch.float64
                r = torch.from_numpy(wl.random_density(1, 4, 32)).to("cuda", dt)
                phi = p.potential(r)
                p.potential(r, phi)                 # graph path
                p.acceleration(phi, coarse_side="flux")
                p.potential_host(r.cpu().numpy())
                del r, phi
    torch.cuda.synchronize()


def test_plans_release_their_memory():
    import torch
    m = nm()
    churn(m, torch, rounds=1)                       # spectra and twiddle caches, graphs
    torch.cuda.empty_cache()
    free0, _ = torch.cuda.mem_get_info()
    churn(m, torch)
    torch.cuda.empty_cache()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 < 64 << 20, (free0 - free1)


@pytest.mark.parametrize("nth", [1, 2, 3, 5])
def test_allocation_failure_is_reported_and_cleaned_up(nth):
    import torch
    m = nm()
    with m.Plan(3, 32, 1.0 / 32) as p:
        p.potential(torch.zeros((3, 32, 32, 32), dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    m.debug_fail_alloc(nth)
    try:
        with pytest.raises(m.NMError) as e:
            m.Plan(3, 32, 1.0 / 32, method="dipole3")
        assert e.value.status == m.NM_ENOMEM
    finally:
        m.debug_fail_alloc(0)
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 < 16 << 20
    # the library still works
    with m.Plan(3, 32, 1.0 / 32, method="dipole3") as p:
        phi = p.potential(torch.from_numpy(wl.random_density(2, 3, 32)).cuda())
        assert torch.isfinite(phi).all()
