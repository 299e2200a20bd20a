"""The allocation-free entry point nm_potential_noalloc, called through the C ABI.

It serves callers that cannot call cudaMalloc while they run (codes whose
device pools are fixed at start-up, processes whose device memory belongs to
another allocator, loops that cannot take cudaMalloc's implicit device-wide
synchronisation).  Its results must match the allocating entry point
nm_potential within the tolerances the other GPU tests use, on consecutive
calls that reuse its single static scratch array.

This file is collected last on purpose, and it also passes alone in a fresh
process.
"""
import ctypes

import numpy as np
import pytest

from paper_2301_06763_gb300 import workloads as wl
from tests.gpu_helpers import FP32_REL_L2, FP32_REL_MAX, FP64_REL_MAX, nm, rel_l2, rel_max

pytestmark = pytest.mark.gpu


def noalloc(opts, rho_t, phi_t):
    import torch
    m = nm()
    f = m.lib().nm_potential_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(m.Options), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return f(ctypes.byref(opts), ctypes.c_void_p(rho_t.data_ptr()), ctypes.c_void_p(phi_t.data_ptr()),
             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def options(L, N, dx0, precision, interp="diagonal"):
    m = nm()
    o = m.Options()
    m.lib().nm_default_options(L, N, dx0, ctypes.byref(o))
    o.precision = m.FP32 if precision == "fp32" else m.FP64
    o.interp = m.DIAGONAL if interp == "diagonal" else m.TRILINEAR
    o.G = 1.3
    return o


@pytest.mark.parametrize("interp", ["trilinear", "diagonal"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_matches_allocating_entry_point_on_consecutive_calls(precision, interp):
    import torch
    m = nm()
    dt = torch.float32 if precision == "fp32" else torch.float64
    # consecutive calls with different sizes: the second reuses (and must fully
    # overwrite) the scratch the first left behind
    for (L, N, seed) in [(3, 16, 1), (2, 32, 2), (3, 16, 3)]:
        dx0 = 0.8 / N
        rho = torch.from_numpy(wl.random_density(seed, L, N)).to("cuda", dt)
        with m.Plan(L, N, dx0, 1.3, precision=precision, interp=interp) as plan:
            ref = plan.potential(rho)
        got = torch.empty_like(ref)
        st = noalloc(options(L, N, dx0, precision, interp), rho, got)
        assert st == m.NM_OK, m.last_error()
        torch.cuda.synchronize()
        a, b = got.cpu().numpy(), ref.cpu().numpy()
        if precision == "fp64":
            assert rel_max(a, b) <= FP64_REL_MAX
        else:
            assert rel_l2(a, b) <= FP32_REL_L2 and rel_max(a, b) <= FP32_REL_MAX


# the extremes of what the fixed array accepts: one level (no restricted
# densities, hole crops or carried holes at all), and the largest FP64 meshes
# of N = 32 that fit with each interpolation (the diagonal rule's carried
# holes need room that the trilinear rule does not, so trilinear fits one
# level more)
@pytest.mark.parametrize("L,N,precision,interp", [
    (1, 16, "fp64", "diagonal"), (1, 32, "fp32", "diagonal"), (1, 32, "fp64", "trilinear"),
    (14, 32, "fp64", "diagonal"), (15, 32, "fp64", "trilinear"), (16, 32, "fp32", "diagonal"),
])
def test_matches_allocating_entry_point_at_the_limits(L, N, precision, interp):
    import torch
    m = nm()
    dt = torch.float32 if precision == "fp32" else torch.float64
    dx0 = 0.8 / N
    with m.Plan(L, N, dx0, 1.3, precision=precision, interp=interp) as plan:
        for seed in (11, 12):      # two calls in a row on the same array
            rho = torch.from_numpy(wl.random_density(seed, L, N)).to("cuda", dt)
            ref = plan.potential(rho)
            got = torch.full_like(ref, float("nan"))
            st = noalloc(options(L, N, dx0, precision, interp), rho, got)
            assert st == m.NM_OK, m.last_error()
            torch.cuda.synchronize()
            a, b = got.cpu().numpy(), ref.cpu().numpy()
            assert np.isfinite(a).all()
            if precision == "fp64":
                assert rel_max(a, b) <= FP64_REL_MAX
            else:
                assert rel_l2(a, b) <= FP32_REL_L2 and rel_max(a, b) <= FP32_REL_MAX


@pytest.mark.parametrize("L,N,precision,interp", [
    (2, 64, "fp64", "diagonal"), (2, 64, "fp32", "trilinear"), (15, 32, "fp64", "diagonal"),
    (16, 32, "fp64", "trilinear"),
])
def test_rejects_meshes_beyond_the_static_maximum(L, N, precision, interp):
    import torch
    m = nm()
    dt = torch.float32 if precision == "fp32" else torch.float64
    rho = torch.zeros((L, N, N, N), dtype=dt, device="cuda")
    phi = torch.full((L, N, N, N), 7.0, dtype=torch.float64, device="cuda")
    st = noalloc(options(L, N, 1.0 / N, precision, interp), rho, phi)
    assert st == m.NM_EINVAL
    assert "NM_NOALLOC_SCRATCH_BYTES" in m.last_error()
    torch.cuda.synchronize()
    assert bool((phi == 7.0).all())      # nothing was launched
