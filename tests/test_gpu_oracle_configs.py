"""The five workload configurations against the FP64 oracle.

Every cell is compared where the oracle's FFT route is affordable (configs 1-3,
and the meshes of N <= 64 in the batch), sampled cells through its direct-sum
route where it is not (the batch's 128^3 meshes, the served 256^3 meshes with 8
levels or more).  Tolerances of the precision pattern:

* FP64 path: relative max error <= 1e-11 (max |Phi_gpu - Phi_oracle| over
  max |Phi_oracle|, all cells of all levels);
* FP32 mode (FP32 transforms and cross-level sums, FP64 spectrum and final
  per-cell addition): relative L2 <= 2e-6 and max <= 1e-5 of max |Phi|.

Where the density has a closed-form potential (Plummer and homogeneous
spheres, a uniform background), the error of the method itself against it
(Eq. 7's measure, per level) is reported too, and the FP32 mode's error must
stay far below it: the reduced precision must not be what limits the answer.

With $NM_ACCURACY_LOG set, the measured errors are appended to that file as one
JSON object per configuration.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2301_06763_gb300 import workloads as wl
from tests import analytic
from tests import oracle_jobs
from tests.gpu_helpers import FP32_REL_L2, FP32_REL_MAX, FP64_REL_MAX, gpu_solve, nm, rel_l2, rel_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    ex = oracle_jobs.spawn_pool()
    yield ex
    ex.shutdown()


def record(config, **kv):
    path = os.environ.get("NM_ACCURACY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"config": config, **kv}) + "\n")


def analytic_errors(w, phi):
    """Per level: max |phi - closed form| / max |closed form| over all levels,
    and the L2 error of the level relative to the closed form's L2."""
    an = [analytic.workload_potential(w, m) for m in range(w.levels)]
    scale = max(np.abs(a).max() for a in an)
    return ([float(np.abs(phi[m] - an[m]).max() / scale) for m in range(w.levels)],
            [float(np.linalg.norm(phi[m] - an[m]) / np.linalg.norm(an[m])) for m in range(w.levels)])


def check_both(ref, got64, got32):
    e = {"fp64_rel_max": rel_max(got64, ref), "fp64_rel_l2": rel_l2(got64, ref),
         "fp32_rel_max": rel_max(got32, ref), "fp32_rel_l2": rel_l2(got32, ref)}
    assert e["fp64_rel_max"] <= FP64_REL_MAX, e
    assert e["fp32_rel_l2"] <= FP32_REL_L2 and e["fp32_rel_max"] <= FP32_REL_MAX, e
    return e


def test_config1_plummer_2x16_every_cell():
    w = wl.config_small()
    rho = w.rho()
    ref = oracle.solve(rho, w.N, w.dx0)
    e = check_both(ref, gpu_solve(rho, w.N, w.dx0), gpu_solve(rho.astype(np.float32), w.N, w.dx0, precision="fp32"))
    disc_max, disc_l2 = analytic_errors(w, ref)
    record(w.name, cells="all", **e, analytic_rel_max_per_level=disc_max, analytic_rel_l2_per_level=disc_l2)


@pytest.mark.parametrize("method", ["original", "dipole"])
def test_config2_binary_4x64_every_cell_and_against_the_closed_form(method, pool):
    # two Plummer spheres and a uniform background: the closed form is the
    # sum of two Plummer potentials and the prism formula over the coarsest
    # cube.  The method's own error against it (discretisation, and the
    # Plummer tails outside the coarsest cube) is 1e-3 .. 4e-2 of max|Phi|
    # per level; the FP32 mode's error against the oracle must be at least a
    # hundred times smaller on every level
    w = wl.config_binary()
    rho = w.rho()
    ref = oracle.solve(rho, w.N, w.dx0, method=method, mapper=pool.map)
    got64 = gpu_solve(rho, w.N, w.dx0, method=method)
    got32 = gpu_solve(rho.astype(np.float32), w.N, w.dx0, precision="fp32", method=method)
    e = check_both(ref, got64, got32)
    disc_max, disc_l2 = analytic_errors(w, ref)
    gpu64_max, _ = analytic_errors(w, got64)
    an = [analytic.workload_potential(w, m) for m in range(w.levels)]
    scale = max(np.abs(a).max() for a in an)
    fp32_per_level = [float(np.abs(got32[m] - ref[m]).max() / scale) for m in range(w.levels)]
    for m in range(w.levels):
        assert abs(gpu64_max[m] - disc_max[m]) <= 1e-9, (m, gpu64_max[m], disc_max[m])
        assert fp32_per_level[m] <= 1e-2 * disc_max[m], (m, fp32_per_level[m], disc_max[m])
    record(w.name + "-" + method, cells="all", **e, analytic_rel_max_per_level=disc_max,
           analytic_rel_l2_per_level=disc_l2, fp32_vs_oracle_rel_max_per_level=fp32_per_level)


def test_config3_contrast_6x128_every_cell(pool):
    # the benchmark mesh: every one of the 6 x 128^3 cells against the FFT
    # oracle (its 11 level convolutions spread over the host cores)
    w = wl.config_contrast()
    rho = w.rho()
    ref = oracle.solve(rho, w.N, w.dx0, mapper=pool.map)
    got64 = gpu_solve(rho, w.N, w.dx0)
    got32 = gpu_solve(rho.astype(np.float32), w.N, w.dx0, precision="fp32")
    e = check_both(ref, got64, got32)
    disc_max, disc_l2 = analytic_errors(w, ref)
    an = [analytic.workload_potential(w, m) for m in range(w.levels)]
    scale = max(np.abs(a).max() for a in an)
    fp32_per_level = [float(np.abs(got32[m] - ref[m]).max() / scale) for m in range(w.levels)]
    for m in range(w.levels):
        assert fp32_per_level[m] <= 1e-2 * disc_max[m], (m, fp32_per_level[m], disc_max[m])
    record(w.name, cells="all", **e, analytic_rel_max_per_level=disc_max, analytic_rel_l2_per_level=disc_l2,
           fp32_vs_oracle_rel_max_per_level=fp32_per_level)


def interface_samples(L, N, rng, extra=1):
    """Cells next to the level interfaces (the coarse side of the finer
    level's region and the fine side of the level's own boundary) on the
    deepest levels, plus random cells."""
    q = N // 4
    out = [(L - 1, 0, N // 2, N - 1), (L - 1, N // 3, 1, N // 2)]
    if L > 1:
        out += [(L - 2, q - 1, N // 2, N // 2), (L - 2, 3 * q, q, q + 1)]
    for _ in range(extra):
        out.append((int(rng.integers(0, L)), *map(int, rng.integers(0, N, 3))))
    return out


def test_config4_batch_of_64_against_the_oracle(pool):
    # the batching configuration solved by one nm_batch_potential call in
    # FP32: every cell of every mesh of N <= 64 against the FFT oracle, and
    # interface and random cells of every 128^3 mesh against the direct sums
    import torch
    m = nm()
    meshes = wl.config_batch(seed=0)
    dens = [w.rho() for w in meshes]
    plans = [m.Plan(w.levels, w.N, w.dx0, precision="fp32") for w in meshes]
    rhos = [torch.from_numpy(r).to("cuda", torch.float32) for r in dens]
    phis = [torch.empty(r.shape, dtype=torch.float64, device="cuda") for r in dens]
    m.batch_potential(plans, rhos, phis)
    torch.cuda.synchronize()
    got = [f.cpu().numpy() for f in phis]
    for p in plans:
        p.close()
    del rhos, phis
    rng = np.random.default_rng(5)
    full_idx = [i for i, w in enumerate(meshes) if w.N <= 64]
    samp_idx = [i for i, w in enumerate(meshes) if w.N == 128]
    samples = {i: interface_samples(meshes[i].levels, meshes[i].N, rng) for i in samp_idx}
    fut_full = {i: pool.submit(oracle_jobs.full_solve, (dens[i], meshes[i].N, meshes[i].dx0, "original", "diagonal"))
                for i in full_idx}
    fut_samp = {i: pool.submit(oracle_jobs.cells, (dens[i], meshes[i].N, meshes[i].dx0, samples[i]))
                for i in samp_idx}
    worst = {"fp32_rel_max": 0.0, "fp32_rel_l2": 0.0, "sampled_rel_max": 0.0}
    for i in full_idx:
        ref = fut_full[i].result()
        a, b = rel_l2(got[i], ref), rel_max(got[i], ref)
        assert a <= FP32_REL_L2 and b <= FP32_REL_MAX, (i, meshes[i].levels, meshes[i].N, a, b)
        worst["fp32_rel_l2"] = max(worst["fp32_rel_l2"], a)
        worst["fp32_rel_max"] = max(worst["fp32_rel_max"], b)
    for i in samp_idx:
        ref = np.asarray(fut_samp[i].result())
        vals = np.array([got[i][c] for c in samples[i]])
        err = float(np.max(np.abs(vals - ref)) / np.max(np.abs(got[i])))
        assert err <= FP32_REL_MAX, (i, meshes[i].levels, err)
        worst["sampled_rel_max"] = max(worst["sampled_rel_max"], err)
    assert len(samp_idx) > 0 and len(full_idx) > 0
    record("batch-64", meshes_every_cell=len(full_idx), meshes_sampled=len(samp_idx),
           sampled_cells=sum(len(s) for s in samples.values()), **worst)


def test_config5_served_stream_against_the_oracle(pool):
    # requests drawn from the serving configuration, including its largest
    # meshes (256^3 with 8 levels or more), served together as one stream in
    # FP32; every small request against the FFT oracle on every cell, the
    # 256^3 ones at interface and random cells against the direct sums
    import torch
    from paper_2301_06763_gb300.serve import Request, Server, run_stream
    nm()
    arrivals = wl.config_serving(rate=300.0, count=400, seed=3)
    big = [(t, w) for (t, w) in arrivals if w.N == 256 and w.levels >= 8][:2]
    small = [(t, w) for (t, w) in arrivals if w.N <= 64][:8]
    chosen = sorted(big + small, key=lambda tw: tw[0])
    assert len(big) == 2
    t0 = chosen[0][0]
    reqs, dens = [], []
    for i, (t, w) in enumerate(chosen):
        r = w.rho()
        dens.append((w, r))
        reqs.append(Request(i, w.levels, w.N, w.dx0, r.astype(np.float32), arrival=t - t0))
    free, _ = torch.cuda.mem_get_info()
    srv = Server(hbm_budget_bytes=int(0.5 * free), slots=4, precision="fp32")
    run_stream(srv, reqs)
    assert len(srv.completed) == len(reqs) and not srv.failed
    srv.close()
    rng = np.random.default_rng(6)
    futs = {}
    for r, (w, rho) in zip(reqs, dens):
        if w.N == 256:
            s = interface_samples(w.levels, w.N, rng, extra=0)
            futs[r.rid] = ("cells", s, pool.submit(oracle_jobs.cells, (rho, w.N, w.dx0, s)))
        else:
            futs[r.rid] = ("full", None, pool.submit(oracle_jobs.full_solve, (rho, w.N, w.dx0, "original", "diagonal")))
    worst = {"fp32_rel_max": 0.0, "fp32_rel_l2": 0.0, "sampled_rel_max": 0.0}
    for r in reqs:
        kind, s, fut = futs[r.rid]
        if kind == "full":
            ref = fut.result()
            a, b = rel_l2(r.result, ref), rel_max(r.result, ref)
            assert a <= FP32_REL_L2 and b <= FP32_REL_MAX, (r.rid, r.levels, r.N, a, b)
            worst["fp32_rel_l2"] = max(worst["fp32_rel_l2"], a)
            worst["fp32_rel_max"] = max(worst["fp32_rel_max"], b)
        else:
            ref = np.asarray(fut.result())
            vals = np.array([r.result[c] for c in s])
            err = float(np.max(np.abs(vals - ref)) / np.max(np.abs(r.result)))
            assert err <= FP32_REL_MAX, (r.rid, r.levels, err)
            worst["sampled_rel_max"] = max(worst["sampled_rel_max"], err)
    record("serving-stream", requests=len(reqs), big=["%dx%d" % (w.levels, w.N) for _, w in big],
           small=["%dx%d" % (w.levels, w.N) for _, w in small], **worst)
