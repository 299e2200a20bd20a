"""The oracle on the paper's test problems at small N: the errors against the
analytic potentials shrink at second order as the grids refine (Sect. 7)."""
import numpy as np

import oracle
from paper_2301_06763_gb300 import workloads as wl
from tests.paper_errors import composite_errors


def test_ellipsoid_errors_converge():
    e = []
    for N in (16, 32):
        w = wl.config_paper_ellipsoid(N=N)
        e.append(composite_errors(w, oracle.solve(w.rho(), w.N, w.dx0)))
    # mean error 1.24 % -> 0.19 % (ratio 6.6; second order gives 4 and the
    # surface staircase improves faster)
    assert e[0]["mean"] / e[1]["mean"] > 4.0
    assert e[1]["max"] < e[0]["max"]
