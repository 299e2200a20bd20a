"""The one-column FP32 z-seam with its spectrum rows staged in shared memory
(schedule pipeline = 0 on FP32 level grids with P = 2N >= 64): the Eq. 11
convolution of the plain one-column kernel, checked against the FP64 oracle on
small meshes for both column-tile widths and against the FP64 GPU path at full
size and against the paired kernel."""
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
@pytest.mark.parametrize("group", [1, 0])
def test_staged_zseam_matches_the_oracle(L, N, tile, group):
    rho = wl.random_density(23 + N, L, N)
    ref = oracle.solve(rho, N, 1.0 / N)
    got = solve(rho.astype(np.float32), N, 1.0 / N, "fp32", (group or L, 16, tile, 0, 0))
    assert rel_l2(got, ref) <= FP32_REL_L2
    assert rel_max(got, ref) <= FP32_REL_MAX


@pytest.mark.parametrize("tile", [0, 1])
def test_staged_zseam_full_size_against_fp64(tile):
    w = wl.config_contrast()
    rho = w.rho()
    a = solve(rho, w.N, w.dx0, "fp64")
    b = solve(rho.astype(np.float32), w.N, w.dx0, "fp32", (w.levels, 16, tile, 0, 0))
    c = solve(rho.astype(np.float32), w.N, w.dx0, "fp32", (w.levels, 16, tile, 2, 0))
    assert rel_l2(b, a) <= FP32_REL_L2
    assert rel_max(b, a) <= FP32_REL_MAX
    assert rel_l2(b, c) <= 1e-6       # the paired kernel: same arithmetic up to FP32 rounding

