"""The FP32 z-seam with two columns per thread (schedule pipeline = 2): the
same Eq. 11 convolution as the one-column kernel, checked against the FP64
oracle on small meshes and against the FP64 GPU path at full size, for both
column-tile widths, and at the largest FFT size (P = 512) against the
one-column kernel and the FP64 path."""
import numpy as np
import pytest

import oracle
from paper_2301_06763_gb300 import workloads as wl
from tests.gpu_helpers import FP32_REL_L2, FP32_REL_MAX, nm, rel_l2, rel_max

pytestmark = pytest.mark.gpu


def solve(rho, N, dx0, precision, sched=None):
    import torch
    m = nm()
    L = rho.shape[0]
    dt = torch.float32 if precision == "fp32" else torch.float64
    with m.Plan(L, N, dx0, precision=precision) as p:
        if sched is not None:
            p.set_schedule(*sched)
            assert p.schedule()["pipeline"] == sched[3]
        r = torch.from_numpy(np.ascontiguousarray(rho)).to("cuda", dt)
        phi = p.potential(r)
        torch.cuda.synchronize()
        return phi.cpu().numpy()


@pytest.mark.parametrize("L,N", [(4, 32), (3, 64)])
@pytest.mark.parametrize("tile", [0, 1])
def test_paired_zseam_matches_the_oracle(L, N, tile):
    rho = wl.random_density(11 + N, L, N)
    ref = oracle.solve(rho, N, 1.0 / N)
    got = solve(rho.astype(np.float32), N, 1.0 / N, "fp32", (L, 16, tile, 2, 0))
    assert rel_l2(got, ref) <= FP32_REL_L2
    assert rel_max(got, ref) <= FP32_REL_MAX


@pytest.mark.parametrize("tile", [0, 1])
def test_paired_zseam_full_size_against_fp64(tile):
    w = wl.config_contrast()
    rho = w.rho()
    a = solve(rho, w.N, w.dx0, "fp64")
    b = solve(rho.astype(np.float32), w.N, w.dx0, "fp32", (w.levels, 16, tile, 2, 0))
    assert rel_l2(b, a) <= FP32_REL_L2
    assert rel_max(b, a) <= FP32_REL_MAX


def test_paired_zseam_largest_fft_size():
    # P = 512: the paired and the one-column kernels agree to FP32 rounding,
    # and both meet the mixed-precision bound against the FP64 path
    L, N = 2, 256
    rho = wl.random_density(5, L, N)
    a = solve(rho, N, 1.0 / N, "fp64")
    one = solve(rho.astype(np.float32), N, 1.0 / N, "fp32", (L, 16, 0, 0, 0))
    two = solve(rho.astype(np.float32), N, 1.0 / N, "fp32", (L, 16, 0, 2, 0))
    assert rel_l2(two, one) <= 1e-6
    for got in (one, two):
        assert rel_l2(got, a) <= FP32_REL_L2
        assert rel_max(got, a) <= FP32_REL_MAX


def test_paired_zseam_schedule_limits():
    import torch
    m = nm()
    with m.Plan(2, 16, 1.0 / 16, precision="fp32") as p:       # P = 32: below the paired kernel's range
        with pytest.raises(m.NMError):
            p.set_schedule(2, 16, 0, 2, 0)
    with m.Plan(2, 32, 1.0 / 32, precision="fp64") as p:       # FP32 only
        with pytest.raises(m.NMError):
            p.set_schedule(2, 16, 0, 2, 0)
    with m.Plan(2, 32, 1.0 / 32, precision="fp32") as p:
        with pytest.raises(m.NMError):
            p.set_schedule(2, 8, 0, 2, 0)                        # 16 values per thread only
        with pytest.raises(m.NMError):
            p.set_schedule(2, 16, 0, 2, 1)                       # not with the fused x/y passes
        p.set_schedule(2, 16, 1, 2, 0)
        r = torch.zeros((2, 32, 32, 32), dtype=torch.float32, device="cuda")
        assert float(p.potential(r).abs().max()) == 0.0


def test_paired_after_one_column_on_one_plan():
    # the spectrum rows over all kx are built when a plan first solves with
    # the paired z-seam, also after solves with the one-column kernel
    import torch
    m = nm()
    L, N = 3, 64
    rho = torch.from_numpy(wl.random_density(2, L, N)).to("cuda", torch.float32)
    with m.Plan(L, N, 1.0 / N, precision="fp32") as p:
        p.set_schedule(L, 16, 0, 0, 0)
        one = p.potential(rho).cpu().numpy()
        p.set_schedule(L, 16, 0, 2, 0)
        two = p.potential(rho).cpu().numpy()
        assert p.spectrum_bytes() >= (N + 1) ** 3 * 20 + (N + 1) ** 2 * 2 * N * 4
    assert rel_l2(two, one) <= 1e-6
