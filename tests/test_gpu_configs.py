"""The batching and serving configurations themselves (not scaled-down
shapes): every mesh of the 64-mesh batch equals its solo solve bit for bit and
sampled cells match the oracle's direct sums; a served request stream drawn
from the serving configuration returns, request by request, what each request
gives alone."""
import numpy as np
import pytest

import oracle
from paper_2301_06763_gb300 import workloads as wl
from tests.gpu_helpers import FP32_REL_MAX, nm

pytestmark = pytest.mark.gpu


def test_batch_config_64_meshes():
    import torch
    m = nm()
    meshes = wl.config_batch(seed=0)
    plans, rhos, phis, dens = [], [], [], []
    for w in meshes:
        rho = w.rho()
        dens.append(rho)
        plans.append(m.Plan(w.levels, w.N, w.dx0, precision="fp32"))
        rhos.append(torch.from_numpy(rho).to("cuda", torch.float32))
        phis.append(torch.empty(rho.shape, dtype=torch.float64, device="cuda"))
    m.batch_potential(plans, rhos, phis)
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    checked = 0
    for i, (w, p, r, f) in enumerate(zip(meshes, plans, rhos, phis)):
        got = f.cpu().numpy()
        assert np.array_equal(got, p.potential(r).cpu().numpy()), i
        if w.N <= 64 and checked < 4:      # a few meshes against the oracle's direct sums
            n = int(rng.integers(0, w.levels))
            cells = [(n, *map(int, rng.integers(0, w.N, 3))) for _ in range(3)]
            ref = oracle.nested_potential_at(dens[i], w.N, w.dx0, cells)
            vals = np.array([got[c] for c in cells])
            assert np.max(np.abs(vals - ref)) <= FP32_REL_MAX * np.max(np.abs(got))
            checked += 1
    assert checked == 4
    for p in plans:
        p.close()


def test_serving_config_stream():
    import torch
    from paper_2301_06763_gb300.serve import Request, Server, run_stream
    m = nm()
    arrivals = wl.config_serving(rate=200.0, count=16, seed=3)
    reqs = []
    for i, (t, w) in enumerate(arrivals):
        reqs.append(Request(i, w.levels, w.N, w.dx0, w.rho().astype(np.float32), arrival=t))
    free, _ = torch.cuda.mem_get_info()
    srv = Server(hbm_budget_bytes=int(0.4 * free), slots=4, precision="fp32")
    run_stream(srv, reqs)
    assert len(srv.completed) == 16 and not srv.failed
    for r in reqs:
        with m.Plan(r.levels, r.N, r.dx0, precision="fp32") as p:
            solo = p.potential(torch.from_numpy(r.rho).cuda()).cpu().numpy()
        assert np.array_equal(r.result, solo), r.rid
    srv.close()
