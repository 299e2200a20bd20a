"""The passes' line transform (fft.cuh) on its own, against the oracle's
radix-2 FFT (itself pinned to the O(n^2) DFT): every size from 8 to 1024
points, both directions, float and double, random lines."""
import numpy as np
import pytest

import oracle
from tests.gpu_helpers import nm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("P", [8, 16, 32, 64, 128, 256, 512, 1024])
@pytest.mark.parametrize("inverse", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_line_transform_matches_oracle_fft(P, inverse, precision):
    import torch
    m = nm()
    rng = np.random.default_rng(P + 7 * inverse)
    lines = 37                                  # more than one CTA's lines, ragged
    x = rng.standard_normal((lines, P)) + 1j * rng.standard_normal((lines, P))
    ref = oracle.fft_axis(x, -1) if not inverse else np.conj(oracle.fft_axis(np.conj(x), -1))
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    d = torch.from_numpy(x).to("cuda", dt)
    m.debug_fft(d, inverse=inverse)
    got = d.cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= (1e-14 if precision == "fp64" else 2e-6), err


def test_bad_sizes_rejected():
    import torch
    m = nm()
    d = torch.zeros((2, 12), dtype=torch.complex64, device="cuda")
    with pytest.raises(m.NMError) as e:
        m.debug_fft(d)
    assert e.value.status == m.NM_EUNSUPPORTED
