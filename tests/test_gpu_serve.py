"""The continuous-batching server: results alone and in the mix, admission by
footprint, and requests that must fail without disturbing the others."""
import numpy as np
import pytest

from paper_2301_06763_gb300 import workloads as wl
from tests.gpu_helpers import nm

pytestmark = pytest.mark.gpu


def requests(n, seed=0, shapes=((2, 8), (3, 16), (2, 32), (4, 16), (3, 8)), spacing=0.0005):
    rng = np.random.default_rng(seed)
    from paper_2301_06763_gb300.serve import Request
    out = []
    for i in range(n):
        L, N = shapes[int(rng.integers(0, len(shapes)))]
        rho = wl.random_density(seed * 1000 + i, L, N).astype(np.float32)
        out.append(Request(i, L, N, 1.0 / N, rho, arrival=i * spacing))
    return out


def solo(r):
    import torch
    m = nm()
    with m.Plan(r.levels, r.N, r.dx0, precision="fp32") as p:
        return p.potential(torch.from_numpy(r.rho).cuda()).cpu().numpy()


def test_same_result_alone_and_in_the_mix():
    from paper_2301_06763_gb300.serve import Server, run_stream
    nm()
    reqs = requests(24)
    srv = Server(hbm_budget_bytes=2 << 30, slots=3, precision="fp32", max_batch=5)
    elapsed, done = run_stream(srv, reqs)
    assert len(done) == 24 and not srv.failed
    assert srv.batches > 1                       # requests joined several batches
    for r in reqs:
        assert np.array_equal(r.result, solo(r))
        assert r.latency is not None and r.latency >= 0
    srv.close()


def test_admission_never_exceeds_the_budget():
    from paper_2301_06763_gb300.serve import Server, run_stream
    m = nm()
    reqs = requests(30, seed=1, spacing=0.0)
    biggest = max(m.footprint_bytes(r.levels, r.N, r.dx0, 1.0, "fp32") + r.levels * r.N ** 3 * 12
                  for r in reqs)
    budget = 2 * biggest
    srv = Server(hbm_budget_bytes=budget, slots=4, precision="fp32")
    run_stream(srv, reqs)
    assert len(srv.completed) == 30
    assert srv.peak_used <= budget
    srv.close()


def test_bad_requests_fail_alone():
    from paper_2301_06763_gb300.serve import Request, Server, run_stream
    nm()
    good = requests(6, seed=2)
    bad_shape = Request(100, 2, 12, 0.1, np.zeros((2, 12, 12, 12), np.float32))   # N not a power of 2
    too_big = Request(101, 8, 256, 1 / 256, np.zeros((1, 1, 1, 1), np.float32))   # over budget
    srv = Server(hbm_budget_bytes=1 << 30, slots=2, precision="fp32")
    run_stream(srv, good + [bad_shape, too_big])
    assert sorted(r.rid for r in srv.failed) == [100, 101]
    assert "budget" in too_big.error and "power of two" in bad_shape.error
    assert len(srv.completed) == 6
    for r in good:
        assert np.array_equal(r.result, solo(r))
    srv.close()


def test_mixed_methods_alone_and_in_the_mix():
    # requests naming the dipole schemes ride in the same batches as plain
    # ones; each result equals the same request solved alone
    import torch
    from paper_2301_06763_gb300.serve import Request, Server, run_stream
    m = nm()
    methods = ["original", "dipole", "dipole3", "dipole3_ds", "dipole3"]
    reqs = []
    for i in range(15):
        L, N = [(3, 8), (4, 16), (3, 16)][i % 3]
        rho = wl.random_density(500 + i, L, N).astype(np.float32)
        reqs.append(Request(i, L, N, 1.0 / N, rho, arrival=i * 0.0003, method=methods[i % len(methods)]))
    srv = Server(hbm_budget_bytes=4 << 30, slots=3, precision="fp32", max_batch=4)
    run_stream(srv, reqs)
    assert len(srv.completed) == 15 and not srv.failed
    for r in reqs:
        with m.Plan(r.levels, r.N, r.dx0, precision="fp32", method=r.method) as p:
            ref = p.potential(torch.from_numpy(r.rho).cuda()).cpu().numpy()
        assert np.array_equal(r.result, ref), r.method
    srv.close()


def test_prewarmed_shapes_allocate_nothing_while_serving():
    # with the request shapes prewarmed, the request loop makes no plan and no
    # buffer (no cudaMalloc, no page-locked allocation) and every result
    # still equals the request solved alone
    from paper_2301_06763_gb300.serve import Server, run_stream
    nm()
    reqs = requests(20, seed=4, spacing=0.001)
    shapes = sorted(set((r.levels, r.N) for r in reqs))
    srv = Server(hbm_budget_bytes=2 << 30, slots=2, precision="fp32", max_batch=1)
    made = srv.prewarm(shapes, per_shape=2)
    assert made == 2 * len(shapes)
    run_stream(srv, reqs)
    assert len(srv.completed) == 20 and not srv.failed
    assert srv.residents_made == made
    for r in reqs:
        assert np.array_equal(r.result, solo(r))
    srv.close()
