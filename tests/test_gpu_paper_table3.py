"""The paper's printed accuracy (Table 3, convolution method, four nested grids
of 128^3): the CUDA FP64 and FP32 paths on the paper's two test problems,
against their analytic potentials (Eq. 7 errors over the composite mesh).

The paper does not state over which cells it averages, so max and mean are
held to 25 % and 30 % of the printed values and the spread to a factor 2.5
(measured on GB300: ellipsoid 0.047 / 0.0034 / 0.0021 %, binary
0.84 / 0.40 / 0.049 %)."""
import os

import numpy as np
import pytest

from paper_2301_06763_gb300 import workloads as wl
from tests.gpu_helpers import gpu_solve
from tests.paper_errors import composite_errors
from tests.test_oracle_green import read_golden

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("problem", ["ellipsoid", "binary"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_reproduces_table3(problem, precision):
    g = read_golden("paper_table3.txt")
    w = (wl.config_paper_ellipsoid if problem == "ellipsoid" else wl.config_paper_binary)(N=128)
    rho = w.rho()
    phi = gpu_solve(rho if precision == "fp64" else rho.astype(np.float32), w.N, w.dx0,
                    precision=precision)
    e = {k: 100.0 * v for k, v in composite_errors(w, phi).items()}
    assert abs(e["max"] - g[problem + "_max"]) <= 0.25 * g[problem + "_max"]
    assert abs(e["mean"] - g[problem + "_mean"]) <= 0.30 * g[problem + "_mean"]
    assert g[problem + "_std"] / 2.5 <= e["std"] <= 2.5 * g[problem + "_std"]
