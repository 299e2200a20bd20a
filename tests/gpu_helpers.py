"""Shared helpers of the GPU tests (import only from tests marked gpu)."""
import functools

import numpy as np


@functools.lru_cache(maxsize=1)
def nm():
    from paper_2301_06763_gb300 import build, nm as _nm
    build.build()
    _nm.lib()
    return _nm


def gpu_solve(rho, N, dx0, G=1.0, precision="fp64", method="original", interp="diagonal"):
    import torch
    m = nm()
    L = rho.shape[0]
    dt = torch.float32 if precision == "fp32" else torch.float64
    with m.Plan(L, N, dx0, G, precision=precision, method=method, interp=interp) as plan:
        r = torch.from_numpy(np.ascontiguousarray(rho)).to("cuda", dt)
        phi = plan.potential(r)
        torch.cuda.synchronize()
        return phi.cpu().numpy()


def rel_max(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


def rel_l2(got, ref):
    return float(np.linalg.norm((got - ref).ravel()) / np.linalg.norm(ref.ravel()))


# Tolerances: FP64 path against the FP64 oracle, and the mixed-precision path
# (FP32 transforms, FP64 spectrum build and final cross-level sum).
FP64_REL_MAX = 1e-11
FP32_REL_L2 = 2e-6
FP32_REL_MAX = 1e-5
