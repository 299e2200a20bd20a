"""The cuFFT baseline that bench.py times beside the library computes the same
level convolution (Sect. 3, Eq. 11) as the oracle, so the comparison is
like for like."""
import numpy as np
import pytest

import oracle
from tests.gpu_helpers import nm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N", [8, 16])
def test_cufft_baseline_equals_oracle_convolution(N):
    import torch
    import bench
    m = nm()
    rng = np.random.default_rng(N)
    M = rng.random((3, N, N, N))
    with m.Plan(1, N, 1.0) as p:
        octant = p.green_octant()
    sh = bench.cufft_half_spectrum(torch, octant, "cuda", torch.float64)
    got = bench.cufft_level_convolutions(torch, torch.from_numpy(M).cuda(), sh).cpu().numpy()
    for f in range(3):
        ref = -oracle.isolated_convolution(M[f], 1.0)      # -(-G/dx) with G = dx = 1
        assert np.max(np.abs(got[f] - ref)) <= 1e-12 * np.max(np.abs(ref))
