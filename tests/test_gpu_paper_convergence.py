"""The paper's convergence and level-count claims on its oblate ellipsoid
(semi-axes 1 : 1 : 0.5 in [-2.25, 2.25]^3), CUDA potential and acceleration
with the carried Eqs. 3-6 interpolation against the closed forms.

* Sect. 7 (Fig. 20, modified method, four levels, N = 16 ... 128): the mean
  errors of Phi and g and the max error of Phi converge at second order, the
  max error of g at first order.  Measured orders (least-squares slope of
  log err against log N): Phi max 1.94, Phi mean 2.84, g max 0.98, g mean
  1.59 -- the last below the printed second order, held to > 1.4.
* Sect. 6 (Fig. 12, original method, N = 128, one to ten levels, errors on
  the x-z plane through the centre): the mean error of Phi falls as levels
  are added, and the errors of g level off instead of growing.  Measured:
  mean Phi error 0.030 % (1 level) down to 0.0025 % (10 levels); max g error
  1.74 % at 3-4 levels and 2.5 % at 10, mean g 0.136 / 0.163 / 0.181 % at
  6 / 8 / 10 levels (the trilinear reading's mean g error grows 8x over the
  same range)."""
import numpy as np
import pytest

from paper_2301_06763_gb300 import workloads as wl
from tests import analytic
from tests.gpu_helpers import nm
from tests.paper_errors import composite_accel_errors, composite_errors

pytestmark = pytest.mark.gpu


def solve_and_accel(w, method, interp, plane=False):
    import torch
    m = nm()
    with m.Plan(w.levels, w.N, w.dx0, precision="fp64", method=method, interp=interp) as p:
        phi = p.potential(torch.from_numpy(w.rho()).cuda())
        g = p.acceleration(phi)
        torch.cuda.synchronize()
        if plane:
            return phi[:, :, w.N // 2, :].cpu().numpy(), g[:, :, :, w.N // 2, :].cpu().numpy()
        return phi.cpu().numpy(), g.cpu().numpy()


def slope(Ns, errs):
    return -np.polyfit(np.log2(Ns), np.log2(errs), 1)[0]


@pytest.mark.parametrize("interp", ["diagonal"])
def test_fig20_convergence_orders(interp):
    Ns = [16, 32, 64, 128]
    pm, pa, gm, ga = [], [], [], []
    for N in Ns:
        w = wl.config_paper_ellipsoid(N=N)
        phi, g = solve_and_accel(w, "dipole", interp)
        ep, eg = composite_errors(w, phi), composite_accel_errors(w, g)
        pm.append(ep["max"]); pa.append(ep["mean"]); gm.append(eg["max"]); ga.append(eg["mean"])
    print("orders: phi max %.2f mean %.2f, g max %.2f mean %.2f" % (slope(Ns, pm), slope(Ns, pa),
                                                                     slope(Ns, gm), slope(Ns, ga)))
    assert slope(Ns, pm) >= 1.7
    assert slope(Ns, pa) >= 1.8
    assert 0.75 <= slope(Ns, gm) <= 1.25
    assert slope(Ns, ga) >= 1.4


def plane_errors(w, phi, g):
    # Eq. 7 errors on the x-z plane y = +dx_m/2 of each level, composite mesh
    N, L = w.N, w.levels
    a, b = N // 4, 3 * N // 4
    comp = w.components[0]
    ep, eg = [], []
    for m in range(L):
        c = wl.level_centres(N, w.dx0, m)
        Z, X = np.meshgrid(c, c, indexing="ij")
        Y = np.full_like(X, c[N // 2])
        an = analytic.oblate_spheroid(X, Y, Z, comp.a, comp.c, comp.rho)
        gan = np.sqrt(sum(v * v for v in analytic.oblate_spheroid_accel(X, Y, Z, comp.a, comp.c, comp.rho)))
        e1 = np.abs((phi[m] - an) / an)
        e2 = np.abs(np.sqrt((g[m] ** 2).sum(axis=0)) - gan) / gan
        mask = np.ones((N, N), bool)
        if m < L - 1 and a <= N // 2 < b:
            mask[a:b, a:b] = False
        ep.append(e1[mask]); eg.append(e2[mask])
    ep, eg = np.concatenate(ep), np.concatenate(eg)
    return ep.mean(), eg.max(), eg.mean()


def test_fig12_errors_versus_level_count():
    ms = [1, 2, 3, 4, 6, 8, 10]
    res = {}
    for m in ms:
        w = wl.config_paper_ellipsoid(N=128, levels=m)
        phi, g = solve_and_accel(w, "original", "diagonal", plane=True)
        res[m] = plane_errors(w, phi, g)
        print(m, ["%.4g" % (100 * v) for v in res[m]])
    phi_mean = [res[m][0] for m in ms]
    assert all(b < a for a, b in zip(phi_mean, phi_mean[1:]))
    assert phi_mean[-1] < phi_mean[0] / 5
    gmax = [res[m][1] for m in ms if m >= 3]
    assert max(gmax) <= 1.6 * gmax[0]
    assert res[10][2] <= 1.5 * res[6][2]
