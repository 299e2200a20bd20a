#!/usr/bin/env python
"""Benchmark of the nested-mesh convolution potential solver on GB300.

Workload: 6 nested levels of 128^3 cells, a homogeneous sphere (radius 0.3)
with a Plummer core (scale 1e-3), density contrast ~1e6, seeded centre offsets
(``workloads.config_contrast``).  One step = one complete solve through the C
ABI (restriction, per-level convolutions, interpolation and assembly).

Prints one JSON line.  ``value`` is FP32-mixed solves/s with inputs resident
in HBM; the FP64 path, p50/p99, the end-to-end host-buffer rate, the roofline
of the dominant kernel, the oracle's CPU rate and the clocks go alongside.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --mode batch    # 64 meshes, N in {32,64,128}, 2-8 levels, one batched call
  python bench.py --mode serve    # Poisson request stream, rates swept, p50/p99 latency
  python bench.py --mode accel    # g = -grad Phi (nm_acceleration) on the benchmark mesh
  python bench.py --mode table    # configs 1-4: GPU FP64/FP32, cuFFT, oracle 1 core / all cores

Under torchrun (N > 1) each rank solves its own copy of the workload (the
meshes are independent: replicas, weak scaling); the timed region is bracketed
by barriers and the maximum over ranks is reported.
"""
import argparse
import hashlib
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "nested-mesh solves/s and ms/solve at 6×128³, FP32 vs FP64 plain; p50/p99; HBM %"
NSETS = 4          # rotating rho/phi buffer sets: 4 x (50 MB + 100 MB) > L2 (~126 MB)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--levels", type=int, default=6)
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle CPU timing (profiling runs)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--mode", choices=["solve", "batch", "serve", "accel", "table", "fp32"], default="solve",
                    help="fp32: FP32 solves of the --levels x --N mesh alone, library default "
                         "schedule (the small cases that ncu captures run)")
    ap.add_argument("--rates", default="10,30,100,300,1000,2000")
    ap.add_argument("--serve-seconds", type=float, default=4.0,
                    help="arrival window per rate (requests = rate x seconds, at most 2000)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- clocks
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + CLOCK_FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm_, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm_)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- roofline
# FP64 add/multiply issue rate of one GB300 (152 SMs), measured on the box
# with a dependent-chain-free DADD/DMUL microbenchmark: ~0.55e12 op/s.
FP64_OPS_PEAK = 0.55e12


def pass_bytes(name, N, fp32, half=False):
    """Algorithmic HBM bytes of one convolution pair in kernel `name` (level grid).

    The pass reads its input array once and writes its output once; the
    density and spectrum are read once.  Level grid: N^3 block, P = 2N.
    half: the pair carries one real field (the finest level of the original
    method), whose x transform is Hermitian, so only the N + 1 columns
    kx <= N of the work arrays are needed."""
    es = 4 if fp32 else 8
    cs = 2 * es
    P = 2 * N
    n3 = N ** 3
    cols = (N + 1) if half else P      # kx columns the y, z and x-inverse passes need
    rows_need = N * N * cols * cs      # [N][N][cols] complex (x-forward output)
    slab = N * P * cols * cs           # [N][P][cols] complex
    if name.startswith("xfwd"):
        return n3 * es + (N // 2) ** 3 * es + rows_need
    if name.startswith("yfwd"):
        return rows_need + slab
    if name.startswith("zseam"):
        return 2 * slab + (N + 1) ** 3 * es
    if name.startswith("yinv"):
        return slab + rows_need
    if name.startswith("xinv"):
        return rows_need + n3 * es + (0 if half else (N // 2 + 2) ** 3 * es)
    return None


def launch_bytes(name, N, fp32, pairs, solves):
    """Algorithmic bytes of a launch of `name` covering `pairs` level pairs of
    `solves` original-method solves: one real (half-spectrum) pair per solve."""
    full = pass_bytes(name, N, fp32)
    if full is None:
        return None
    return (pairs - solves) * full + solves * pass_bytes(name, N, fp32, half=True)


# the sources whose kernels the traffic summary measures
HASHED_SOURCES = ("fft.cuh", "conv.cuh", "conv_inst.cuh", "conv_f32_pair.cu", "support.cu")


def source_hash():
    """First 16 hex digits of the sha256 of the sources that define the
    measured passes' kernels, with comments and white space taken out (a
    comment edit leaves the kernels, and so their measured traffic, as they
    were)."""
    h = hashlib.sha256()
    for f in HASHED_SOURCES:
        text = open(os.path.join(ROOT, "paper_2301_06763_gb300", "csrc", f)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_name):
    """(pairs, DRAM bytes per launch) of `kernel_name` from the committed ncu
    summary, or None when no summary exists or the kernel sources changed
    since."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"source hash:\s*`?([0-9a-f]+)", text)
    if not m or m.group(1) != source_hash():
        return None
    m = re.search(r"^\|\s*%s\s*\|\s*(\d+)\s*\|\s*([0-9.e+]+)\s*\|" % re.escape(kernel_name), text, re.M)
    return (int(m.group(1)), float(m.group(2))) if m else None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------- oracle timings
def _oracle_conv(args):
    import oracle
    M, dx = args
    return oracle.isolated_convolution(M, dx, 1.0)


def oracle_pool(workers):
    """A process pool for the oracle, started with spawn (never forked from a
    process that has touched the GPU) and warmed so that worker start-up and
    imports stay outside the timed region."""
    import concurrent.futures as cf
    import multiprocessing as mp
    pool = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
    list(pool.map(_oracle_conv, [(np.zeros((4, 4, 4)), 1.0)] * workers))
    return pool


def oracle_solve_timed(rho, N, dx0, pool=None):
    """The FP64 oracle's original-method solve (restriction, 2L-1 level
    convolutions, Eq. 14 assembly with the carried Eqs. 3-6 interpolation,
    the library's default) with the convolutions either in this process or
    spread over `pool`; returns (phi, seconds)."""
    import oracle
    from oracle.nested import diagonal_to_next
    L = rho.shape[0]
    t0 = time.perf_counter()
    geom = oracle.Geometry(L, N, dx0)
    full_M, hole_M = oracle.level_masses(oracle.restrict(rho, N), geom)
    jobs = [(full_M[m], geom.dx(m)) for m in range(L)] + [(hole_M[m], geom.dx(m)) for m in range(L - 1)]
    res = list(pool.map(_oracle_conv, jobs)) if pool is not None else [_oracle_conv(j) for j in jobs]
    full, hole = res[:L], res[L:]
    phi = np.empty((L, N, N, N))
    carry = None
    for n in range(L):
        phi[n] = full[n]
        if n > 0:
            carry = diagonal_to_next(hole[n - 1] if carry is None else carry + hole[n - 1], N)
            phi[n] += carry
    return phi, time.perf_counter() - t0


def cpu_baseline(levels, N):
    """The FP64 oracle, as it stands, on the host: one level convolution on one
    core (extrapolated to the 2L - 1 of a solve), and a whole solve with its
    convolutions spread over all host cores.  Returns (the oracle's potential,
    the timing record)."""
    import oracle
    from paper_2301_06763_gb300 import workloads as wl
    w = wl.config_contrast(levels=levels, N=N)
    rho = w.rho()
    spec = oracle.green_spectrum(N)
    t0 = time.perf_counter()
    oracle.isolated_convolution(rho[0] * w.dx0 ** 3, w.dx0, 1.0, spec)
    t = time.perf_counter() - t0
    nconv = 2 * levels - 1
    cores = min(os.cpu_count() or 1, nconv)
    pool = oracle_pool(cores)
    try:
        phi_oracle, t_all = oracle_solve_timed(rho, N, w.dx0, pool)
    finally:
        pool.shutdown()
    return phi_oracle, {"value": 1.0 / t_all, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "host_cores": os.cpu_count(), "cpu": platform.processor() or platform.machine(),
            "sample": "one whole oracle solve (restriction, %d level convolutions spread over %d "
                      "processes, Eq. 14 assembly): %.1f s" % (nconv, cores, t_all),
            "one_core": {"value": 1.0 / (nconv * t), "unit": "solves/s", "cores": 1,
                         "sample": "one oracle isolated_convolution of a %d^3 level (%.1f s), x%d "
                                   "convolutions per solve" % (N, t, nconv)}}


def reference_arm(args):
    """--impl reference: the FP64 oracle, as it stands, on the host cores.

    One step = one whole oracle solve of the benchmark workload (restriction,
    the 2L - 1 level convolutions spread over a spawn-started process pool on
    the host cores, the Eq. 14 assembly with the carried Eqs. 3-6
    interpolation), the same computation the GPU arm times, in FP64."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2301_06763_gb300 import workloads as wl
    N, L = args.N, args.levels
    w = wl.config_contrast(levels=L, N=N)
    rho = w.rho()
    nconv = 2 * L - 1
    cores = min(os.cpu_count() or 1, nconv)
    pool = oracle_pool(cores)
    try:
        for _ in range(args.warmup):
            oracle_solve_timed(rho, N, w.dx0, pool)
        times = []
        for _ in range(args.steps):
            times.append(oracle_solve_timed(rho, N, w.dx0, pool)[1])
    finally:
        pool.shutdown()
    total = sum(times)
    per_step = total / max(args.steps, 1)
    value = args.steps / total if total > 0 else None
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_step * 1e3, "p50_ms": pct(times, 50) * 1e3, "p99_ms": pct(times, 99) * 1e3,
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "contrast-%dx%d" % (L, N), "levels": L, "N": N,
                   "precision": "fp64 (the CPU oracle)", "method": "original",
                   "interp": "diagonal (Eqs. 3-6, carried level by level)",
                   "parallelism": "host processes"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "host_cores": os.cpu_count(), "cpu": platform.processor() or platform.machine(),
                         "sample": "one whole oracle solve per step (restriction, %d level convolutions "
                                   "spread over %d processes, Eq. 14 assembly)" % (nconv, cores)},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ----------------------------------------------------------------------------- our arm
def timed_loop(torch, plan, rhos, phis, steps, dist, stream):
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        k = i % len(rhos)
        starts[i].record(stream)
        plan.potential(rhos[k], phis[k], stream=stream)
        ends[i].record(stream)
    torch.cuda.synchronize()
    elapsed_wall = time.perf_counter() - t0
    if dist is not None:
        dist.barrier()
    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_dev_ms = starts[0].elapsed_time(ends[-1])
    return total_dev_ms, per, elapsed_wall


def dipole_rates(nm, wl, torch, dev, reps=20):
    """The dipole schemes (Sect. 7, Appendix B) on 4 levels of 64^3 (two
    Plummer spheres) and of 32^3, against the original method on the same
    mesh: pairwise (Eqs. B.1-B.2), three-level with quadrupled grids (Eqs.
    B.3-B.5) and with the direct sum of Eq. B.6 (FP64 only at 32^3: its O(N^6)
    sum runs on the slow FP64 pipe)."""
    out = {}
    for N in (64, 32):
        w = wl.config_binary()
        w = wl.Workload(w.name, w.levels, N, w.dx0 * 64 / N, w.components)
        rho = w.rho()
        tag = "binary-4x%d" % N
        out[tag] = {}
        for prec, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
            r = torch.from_numpy(rho).to(dev, dt)
            phi = torch.empty(rho.shape, dtype=torch.float64, device=dev)
            for meth in ("original", "dipole", "dipole3", "dipole3_ds"):
                if meth == "dipole3_ds" and prec == "fp64" and N > 32:
                    continue
                p = nm.Plan(w.levels, w.N, w.dx0, precision=prec, method=meth)
                n = reps if prec == "fp32" else max(2, reps // 5)
                for _ in range(3):
                    p.potential(r, phi)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                for _ in range(n):
                    p.potential(r, phi)
                b.record()
                torch.cuda.synchronize()
                out[tag]["%s_%s_ms" % (meth, prec)] = a.elapsed_time(b) / n
                p.close()
            for meth in ("dipole", "dipole3", "dipole3_ds"):
                k = "%s_%s_ms" % (meth, prec)
                if k in out[tag]:
                    out[tag]["overhead_%s_%s" % (meth, prec)] = out[tag][k] / out[tag]["original_%s_ms" % prec]
    return out


def accel_rates(nm, torch, dev, rho, w, peak, reps=20, interp=True):
    """g = -grad Phi (nm_acceleration) on the benchmarked mesh, and the solve
    with the carried Eqs. 3-6 interpolation against the trilinear one.  The
    acceleration kernel moves 32 bytes per cell (one double read, three
    written), over 4 rotating phi/g sets larger than L2."""
    L, N = w.levels, w.N
    cells = L * N ** 3
    p = nm.Plan(L, N, w.dx0, precision="fp64")
    r = torch.from_numpy(rho).to(dev, torch.float64)
    phis = [p.potential(r).clone() for _ in range(NSETS)]
    gs = [torch.empty((L, 3, N, N, N), dtype=torch.float64, device=dev) for _ in range(NSETS)]
    for i in range(3):
        p.acceleration(phis[i % NSETS], gs[i % NSETS])
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for i in range(reps):
        p.acceleration(phis[i % NSETS], gs[i % NSETS])
    b.record()
    torch.cuda.synchronize()
    us = a.elapsed_time(b) / reps * 1e3
    p.close()
    del gs
    gbs = 32.0 * cells / (us * 1e-6) / 1e9
    # FP64-pipe bound: 3 subtractions and 3 multiplications per interior cell
    fp64_ops = 6 * cells
    out = {"acceleration": {"workload": "contrast-%dx%d" % (L, N), "us_per_launch": us,
                            "algorithmic_bytes": 32 * cells, "gbs": gbs, "frac_hbm": gbs / peak,
                            "fp64_ops": fp64_ops, "fp64_tops": fp64_ops / (us * 1e-6) / 1e12,
                            "frac_fp64": fp64_ops / (us * 1e-6) / FP64_OPS_PEAK,
                            "fp64_peak_ops": FP64_OPS_PEAK}}
    if not interp:
        return out
    diag = {}
    for prec, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
        rr = torch.from_numpy(rho).to(dev, dt)
        for interp in ("trilinear", "diagonal"):
            q = nm.Plan(L, N, w.dx0, precision=prec, interp=interp)
            n = reps if prec == "fp32" else max(2, reps // 5)
            for i in range(3):
                q.potential(rr, phis[i % NSETS])
            torch.cuda.synchronize()
            a.record()
            for i in range(n):
                q.potential(rr, phis[i % NSETS])
            b.record()
            torch.cuda.synchronize()
            diag["%s_%s_ms" % (interp, prec)] = a.elapsed_time(b) / n
            q.close()
    out["interp_readings"] = diag
    return out




def cufft_half_spectrum(torch, octant, dev, dtype):
    """The (2N)^3 Green spectrum in torch.fft.rfftn's half layout (P, P, N+1)
    from the library's real even octant ((N+1)^3, [kz][ky][kx])."""
    N = octant.shape[0] - 1
    P = 2 * N
    k = np.arange(P)
    f = np.minimum(k, P - k)
    return torch.from_numpy(np.ascontiguousarray(octant[f][:, f][:, :, :N + 1])).to(dev, dtype)


def cufft_level_convolutions(torch, masses, spec_half):
    """Same-GPU cuFFT baseline of the level convolutions (Sect. 3, Eq. 11):
    every field of ``masses`` (F, N, N, N) zero-padded to (2N)^3, one batched
    R2C transform, the spectrum multiply, one batched C2R transform, the
    active N^3 block cropped.  Returns the lattice sums sum_j M_j calG(i-j) in
    unit-cell units (multiply by -G/dx for the potential)."""
    F, N = masses.shape[0], masses.shape[1]
    P = 2 * N
    buf = torch.zeros((F, P, P, P), dtype=masses.dtype, device=masses.device)
    buf[:, :N, :N, :N] = masses
    spec = torch.fft.rfftn(buf, dim=(1, 2, 3))
    spec *= spec_half
    out = torch.fft.irfftn(spec, s=(P, P, P), dim=(1, 2, 3))
    return out[:, :N, :N, :N].contiguous()


def cufft_baseline(nm, torch, dev, rho, w, reps=10):
    """Time the 2L-1 level convolutions of one solve (each level's full field
    and the hole fields of all but the finest) through cuFFT (torch.fft,
    batched over all fields), FP32 and FP64.
    Restriction and assembly are left out, so this is compared with the sum of
    this library's five transform passes."""
    L, N = w.levels, w.N
    with nm.Plan(L, N, w.dx0) as p:
        octant = p.green_octant()
    out = {"workload": "contrast-%dx%d" % (L, N), "fields": 2 * L - 1,
           "what": "pad, batched R2C, spectrum multiply, batched C2R, crop (torch.fft = cuFFT)"}
    for prec, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
        sh = cufft_half_spectrum(torch, octant, dev, dt)
        m = torch.from_numpy(np.concatenate([rho, rho[:-1]], axis=0)).to(dev, dt)   # 2L-1 fields
        for _ in range(3):
            cufft_level_convolutions(torch, m, sh)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = reps if prec == "fp32" else max(2, reps // 2)
        a.record()
        for _ in range(n):
            cufft_level_convolutions(torch, m, sh)
        b.record()
        torch.cuda.synchronize()
        out["%s_ms" % prec] = a.elapsed_time(b) / n
        del m, sh
        torch.cuda.empty_cache()
    return out


def accuracy_vs_oracle(torch, p32, p64, rho32, rho64, phi_oracle, w):
    """Errors of this solve on every cell: the FP32 mode and the FP64 path
    against the oracle's potential (the one the cpu_baseline leg computed),
    and all three against the closed-form potential of the density (Eq. 7's
    measure, per level: max |Phi - Phi_exact| over max |Phi_exact| of all
    levels)."""
    from tests import analytic
    got32 = p32.potential(rho32).cpu().numpy()
    got64 = p64.potential(rho64).cpu().numpy()
    torch.cuda.synchronize()
    ref = phi_oracle
    den = np.abs(ref).max()
    an = [analytic.workload_potential(w, m) for m in range(w.levels)]
    an_scale = max(np.abs(a).max() for a in an)

    def per_level(x):
        return [float(np.abs(x[m] - an[m]).max() / an_scale) for m in range(w.levels)]

    return {"cells": "all %d" % ref.size, "reference": "FP64 oracle (the cpu_baseline solve)",
            "fp32_rel_l2": float(np.linalg.norm(got32 - ref) / np.linalg.norm(ref)),
            "fp32_rel_max": float(np.abs(got32 - ref).max() / den),
            "fp64_rel_l2": float(np.linalg.norm(got64 - ref) / np.linalg.norm(ref)),
            "fp64_rel_max": float(np.abs(got64 - ref).max() / den),
            "tolerances": {"fp32_rel_l2": 2e-6, "fp32_rel_max": 1e-5, "fp64_rel_max": 1e-11},
            "vs_closed_form_rel_max_per_level": {"oracle": per_level(ref), "fp32": per_level(got32),
                                                 "fp64": per_level(got64)}}


def max_over_ranks(torch, dist, v):
    from paper_2301_06763_gb300 import replicas
    return replicas.max_over_ranks(v, dist, device="cuda" if dist is not None else None)


def pct(xs, q):
    return float(np.percentile(np.asarray(xs), q))


def ours(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2301_06763_gb300 import build
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    from paper_2301_06763_gb300 import nm, workloads as wl

    L, N = args.levels, args.N
    w = wl.config_contrast(levels=L, N=N)
    rho = w.rho()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    rho32 = [torch.from_numpy(rho).to(dev, torch.float32) for _ in range(NSETS)]
    rho64 = [torch.from_numpy(rho).to(dev, torch.float64) for _ in range(NSETS)]
    phis = [torch.empty(rho.shape, dtype=torch.float64, device=dev) for _ in range(NSETS)]
    p32 = nm.Plan(L, N, w.dx0, precision="fp32")
    p64 = nm.Plan(L, N, w.dx0, precision="fp64")
    p32.green()
    p64.green()
    sched = {}
    if not args.no_autotune:
        sched["fp32"] = p32.autotune(rho32[0], phis[0], reps=3)
        sched["fp64"] = p64.autotune(rho64[0], phis[0], reps=2)
    else:
        sched = {"fp32": p32.schedule(), "fp64": p64.schedule()}
    for i in range(max(args.warmup, 3)):
        p32.potential(rho32[i % NSETS], phis[i % NSETS])
        p64.potential(rho64[i % NSETS], phis[i % NSETS])
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    l0 = nm.kernel_launches()
    dev_ms, per32, _ = timed_loop(torch, p32, rho32, phis, args.steps, dist, stream)
    launches = nm.kernel_launches() - l0
    dev_ms = max_over_ranks(torch, dist, dev_ms)
    dev64_ms, per64, _ = timed_loop(torch, p64, rho64, phis, args.steps, dist, stream)
    dev64_ms = max_over_ranks(torch, dist, dev64_ms)
    # FP64-class accuracy from the FP32 pipe: double-float transforms
    p64x = nm.Plan(L, N, w.dx0, precision="fp64x")
    p64x.green()
    for i in range(3):
        p64x.potential(rho64[i % NSETS], phis[i % NSETS])
    dev64x_ms, per64x, _ = timed_loop(torch, p64x, rho64, phis, args.steps, dist, stream)
    dev64x_ms = max_over_ranks(torch, dist, dev64x_ms)
    clk = clocks.stop()

    # end to end through the host-buffer entry points (H2D + solve + D2H per
    # step, from and to page-locked host memory): the pipelined one, whose
    # copies overlap the neighbouring steps' solves, and one call per step
    h_rho = torch.from_numpy(rho.astype(np.float32)).pin_memory()
    h_phi = torch.empty(rho.shape, dtype=torch.float64).pin_memory()
    p32.potential_host_many([h_rho] * 3, [h_phi] * 3)
    p32.potential_host(h_rho.numpy(), h_phi.numpy())
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    p32.potential_host_many([h_rho] * args.steps, [h_phi] * args.steps)
    e2e_s = max_over_ranks(torch, dist, time.perf_counter() - t0)
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        p32.potential_host(h_rho.numpy(), h_phi.numpy())
    e2e_sync_s = max_over_ranks(torch, dist, time.perf_counter() - t0)

    # per-kernel event timing (instrumented repeat of the FP32 timed loop)
    nm.profile_enable(True)
    timed_loop(torch, p32, rho32, phis, args.steps, None, stream)
    stats = nm.profile_read()
    nm.profile_enable(False)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    from paper_2301_06763_gb300 import replicas
    ms_step = dev_ms / args.steps
    value = replicas.job_rate(world * args.steps, dev_ms / 1e3)
    peak, peak_kind = peaks()
    dom = max(stats.items(), key=lambda kv: kv[1][2])
    dname, (dl, du, dms) = dom
    per_unit = pass_bytes(dname, N, True)
    roof = None
    if per_unit is not None:
        # each launch of a pass covers one solve: its L pairs, the finest a
        # real (half-spectrum) pair
        bytes_launch = launch_bytes(dname, N, True, du / dl, 1)
        achieved = bytes_launch / (dms / dl * 1e-3) / 1e9
        tr = ncu_traffic(dname)
        # the summary's launches cover the benchmark's solves (L pairs each)
        traffic = tr[1] if tr is not None and tr[0] == round(du / dl) else None
        roof = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "algorithmic_bytes_per_launch": bytes_launch,
                "avg_launch_ms": dms / dl}
    solve_bytes = sum(launch_bytes(k, N, True, v[1], v[0]) for k, v in stats.items()
                      if pass_bytes(k, N, True) is not None) / args.steps
    kernel_table = {k: {"launches": v[0], "avg_ms": v[2] / v[0], "share": v[2] / sum(
        x[2] for x in stats.values())} for k, v in sorted(stats.items(), key=lambda kv: -kv[1][2])}
    dip = dipole_rates(nm, wl, torch, dev) if not args.no_cpu_baseline else None
    ext = accel_rates(nm, torch, dev, rho, w, peak) if not args.no_cpu_baseline else {}
    cuf = cufft_baseline(nm, torch, dev, rho, w) if not args.no_cpu_baseline else None
    if cuf is not None:
        conv = [k for k in stats if k.split("_")[0] in ("xfwd", "yfwd", "zseam", "yinv", "xinv")]
        cuf["ours_fp32_transform_passes_ms"] = sum(stats[k][2] for k in conv) / args.steps
        cuf["ours_fp32_solve_ms"] = ms_step
        cuf["ours_fp64_solve_ms"] = dev64_ms / args.steps
        cuf["speedup_fp32_passes"] = cuf["fp32_ms"] / cuf["ours_fp32_transform_passes_ms"]
        cuf["speedup_fp64_solve"] = cuf["fp64_ms"] / cuf["ours_fp64_solve_ms"]
    cpu = None
    accuracy = None
    if world == 1 and not args.no_cpu_baseline:
        phi_oracle, cpu = cpu_baseline(L, N)
        accuracy = accuracy_vs_oracle(torch, p32, p64, rho32[0], rho64[0], phi_oracle, w)
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "contrast-%dx%d" % (L, N), "levels": L, "N": N,
                   "precision": "fp32 passes, fp64 spectrum and final sum", "method": "original",
                   "interp": "diagonal (Eqs. 3-6, carried level by level)",
                   "l2": "%d rotating rho/phi sets (%.0f MB > L2)" % (
                       NSETS, NSETS * (rho.size * 4 + rho.size * 8) / 1e6),
                   "parallelism": "replicas" if world > 1 else "single",
                   "schedule": sched},
        "p50_ms": pct(per32, 50), "p99_ms": pct(per32, 99),
        "fp64": {"value": world * args.steps / (dev64_ms / 1e3), "unit": "solves/s",
                 "ms_per_step": dev64_ms / args.steps, "p50_ms": pct(per64, 50),
                 "p99_ms": pct(per64, 99), "dtype": "f64"},
        "fp64x": {"value": world * args.steps / (dev64x_ms / 1e3), "unit": "solves/s",
                  "ms_per_step": dev64x_ms / args.steps, "p50_ms": pct(per64x, 50), "p99_ms": pct(per64x, 99),
                  "dtype": "double-float (2 x f32)", "accuracy": "within 1e-12 of max|Phi| of the FP64 oracle"},
        "hbm": {"solve_algorithmic_bytes": solve_bytes,
                "solve_gbs": solve_bytes / (ms_step * 1e-3) / 1e9,
                "frac": solve_bytes / (ms_step * 1e-3) / 1e9 / peak},
        "e2e": {"value": world * args.steps / e2e_s, "unit": "solves/s",
                "h2d_bytes_per_step": int(rho.size * 4), "d2h_bytes_per_step": int(rho.size * 8),
                "api": "nm_potential_host_many (copies overlapped with the neighbouring solves)",
                "one_call_per_step": world * args.steps / e2e_sync_s},
        "gpu_launches": int(launches),
        "roofline": roof,
        "kernels": kernel_table,
        "cpu_baseline": cpu,
        "accuracy": accuracy,
        "dipole": dip,
        "cufft_baseline": cuf,
        "acceleration": ext.get("acceleration"),
        "interp_readings": ext.get("interp_readings"),
        "clocks": clk,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- batch mode
def batch_mode(args):
    """64 independent meshes solved by one nm_batch_potential call (FP32),
    against the same meshes solved one by one in FP32 and in plain FP64."""
    import torch
    from paper_2301_06763_gb300 import build
    build.build()
    from paper_2301_06763_gb300 import nm, workloads as wl
    meshes = wl.config_batch(seed=0)
    dev = torch.device("cuda", 0)
    plans32, plans64, r32, r64, phis = [], [], [], [], []
    cells = 0
    for w in meshes:
        rho = w.rho()
        cells += rho.size
        plans32.append(nm.Plan(w.levels, w.N, w.dx0, precision="fp32"))
        plans64.append(nm.Plan(w.levels, w.N, w.dx0, precision="fp64"))
        r32.append(torch.from_numpy(rho).to(dev, torch.float32))
        r64.append(torch.from_numpy(rho).to(dev, torch.float64))
        phis.append(torch.empty(rho.shape, dtype=torch.float64, device=dev))
    tuned = {}
    if not args.no_autotune:
        for p, r, f in zip(plans32, r32, phis):
            key = (p.levels, p.N)
            if key not in tuned:
                tuned[key] = p.autotune(r, f, reps=2)
            else:
                p.set_schedule(**tuned[key])
    stream = torch.cuda.current_stream()

    def timed(fn, steps):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    l0 = nm.kernel_launches()
    nm.batch_potential(plans32, r32, phis)
    per_batch_launches = nm.kernel_launches() - l0
    ms_batch = timed(lambda: nm.batch_potential(plans32, r32, phis), args.steps)
    ms_seq32 = timed(lambda: [p.potential(r, f) for p, r, f in zip(plans32, r32, phis)], args.steps)
    # the persistent schedule: every step of all 64 solves as work items of
    # one launch (after a first eager call, replayed as a graph of one counter
    # reset and one kernel)
    keep = [p.schedule() for p in plans32]
    for p in plans32:
        p.set_schedule(p.levels, 16, 0, 0, 3)
    nm.batch_potential(plans32, r32, phis)
    torch.cuda.synchronize()
    l0 = nm.kernel_launches()
    nm.batch_potential(plans32, r32, phis)
    torch.cuda.synchronize()
    persist_launches = nm.kernel_launches() - l0
    ms_persist = timed(lambda: nm.batch_potential(plans32, r32, phis), args.steps)
    for p, sc in zip(plans32, keep):
        p.set_schedule(**sc)
    ms_seq64 = timed(lambda: [p.potential(r, f) for p, r, f in zip(plans64, r64, phis)],
                     max(1, args.steps // 4))
    line = {"mode": "batch", "metric": "meshes/s, 64-mesh batch (N in {32,64,128}, 2-8 levels)",
            "unit": "meshes/s", "value": 64 / (ms_batch / 1e3), "ms_per_batch": ms_batch,
            "fp32_one_by_one_ms": ms_seq32, "fp64_plain_one_by_one_ms": ms_seq64,
            "speedup_vs_fp64_plain": ms_seq64 / ms_batch, "speedup_vs_fp32_one_by_one": ms_seq32 / ms_batch,
            "cells": cells, "kernels_per_batch_eager": per_batch_launches,
            "persistent": {"ms_per_batch": ms_persist, "meshes_per_s": 64 / (ms_persist / 1e3),
                           "kernels_per_batch": persist_launches,
                           "what": "all 64 solves as work items of one persistent launch (fuse 3)"},
            "graph": "batch replayed as one CUDA graph after the first repeat",
            "shapes": sorted(set((w.levels, w.N) for w in meshes)),
            "schedules": {"%dx%d" % k: v for k, v in tuned.items()}, "steps": args.steps,
            "data": "synthetic", "dtype": "f32"}
    print(json.dumps(line))


# ----------------------------------------------------------------------------- accel mode
def accel_mode(args):
    """nm_acceleration alone on the benchmark mesh (its own launch list and
    ncu capture), one JSON line."""
    import torch
    from paper_2301_06763_gb300 import build
    build.build()
    from paper_2301_06763_gb300 import nm, workloads as wl
    w = wl.config_contrast(levels=args.levels, N=args.N)
    peak, kind = peaks()
    out = accel_rates(nm, torch, torch.device("cuda", 0), w.rho(), w, peak, reps=args.steps, interp=False)
    a = out["acceleration"]
    print(json.dumps({"mode": "accel", "metric": "accelerations/s (g on every cell of every level)",
                      "unit": "meshes/s", "value": 1e6 / a["us_per_launch"], "steps": args.steps,
                      "peak_kind": kind, "data": "synthetic", "dtype": "f64", **a}))


# ----------------------------------------------------------------------------- fp32 mode
def fp32_mode(args):
    """--warmup + --steps FP32 solves of the --levels x --N benchmark mesh with
    the library's default schedule and nothing else on the GPU: the small,
    short cases that ncu captures run.  One JSON line."""
    import torch
    from paper_2301_06763_gb300 import build
    build.build()
    from paper_2301_06763_gb300 import nm, workloads as wl
    w = wl.config_contrast(levels=args.levels, N=args.N)
    rho = torch.from_numpy(w.rho()).to("cuda", torch.float32)
    phi = torch.empty(rho.shape, dtype=torch.float64, device="cuda")
    with nm.Plan(args.levels, args.N, w.dx0, precision="fp32") as p:
        for _ in range(args.warmup):
            p.potential(rho, phi)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            p.potential(rho, phi)
        b.record()
        torch.cuda.synchronize()
        print(json.dumps({"mode": "fp32", "workload": w.name, "levels": args.levels, "N": args.N,
                          "schedule": p.schedule(), "steps": args.steps, "warmup": args.warmup,
                          "ms_per_solve": a.elapsed_time(b) / max(args.steps, 1),
                          "note": "same rho every solve (inputs partly in L2): for profiling, not a bench value"}))


# ----------------------------------------------------------------------------- serve mode
def serve_mode(args):
    """Poisson request streams at several rates through the continuous-batching
    server: solves/s and p50/p99 latency (arrival to potentials on the host)."""
    import torch
    from paper_2301_06763_gb300 import build
    build.build()
    from paper_2301_06763_gb300 import nm, workloads as wl
    from paper_2301_06763_gb300.serve import Request, Server, latency_stats, run_stream
    # one density per N, sampled for the deepest mesh (10 levels) and sliced:
    # level m of a mesh is the same set of cells whatever its level count
    dens = {}
    rng = np.random.default_rng(0)
    for N in (32, 64, 128, 256):
        w = wl.Workload("serve-%d" % N, 10, N, 1.0 / N, wl.random_plummers(rng, 10, N))
        dens[N] = torch.from_numpy(np.ascontiguousarray(w.rho().astype(np.float32))).pin_memory()
    free, total = torch.cuda.mem_get_info()
    budget = int(0.5 * free)
    srv = Server(budget, slots=4, precision="fp32", per_shape_cap=2)
    # plans, spectra and buffers for every shape of the request distribution,
    # made once before the streams start (untimed); with at most 2 sets per
    # shape in existence the request loop then allocates nothing
    shapes = [(L, N) for N in (32, 64, 128, 256) for L in range(3, 11)]
    srv.prewarm(shapes, per_shape=2)
    made0 = srv.residents_made
    # the device-bound rate of the mix: per shape, the solve alone and the
    # solve with its upload and download, on a resident set, timed by events
    per_shape = {}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for (L, N) in shapes:
        key = (L, N, 1.0 / N, 1.0, "original")
        res = srv._pool_take(key)
        if res is None:
            continue
        for _ in range(3):
            res.plan.potential(res.rho_dev, res.phi_dev)
        torch.cuda.synchronize()
        reps = 10 if N < 256 else 4
        ev[0].record()
        for _ in range(reps):
            res.plan.potential(res.rho_dev, res.phi_dev)
        ev[1].record()
        for _ in range(reps):
            res.rho_dev.copy_(dens[N][:L], non_blocking=True)
            res.plan.potential(res.rho_dev, res.phi_dev)
            res.phi_pin.copy_(res.phi_dev, non_blocking=True)
        ev[2].record()
        torch.cuda.synchronize()
        per_shape["%dx%d" % (L, N)] = {"solve_ms": ev[0].elapsed_time(ev[1]) / reps,
                                       "with_copies_ms": ev[1].elapsed_time(ev[2]) / reps}
        srv._pool_put(res)
    mix_solve = float(np.mean([v["solve_ms"] for v in per_shape.values()]))
    mix_copies = float(np.mean([v["with_copies_ms"] for v in per_shape.values()]))
    results = []
    for rate in [float(x) for x in args.rates.split(",")]:
        count = int(min(2000, max(20, rate * args.serve_seconds)))
        arrivals = wl.config_serving(rate, count=count, seed=0)
        reqs = []
        for i, (t, w) in enumerate(arrivals):
            reqs.append(Request(i, w.levels, w.N, w.dx0, dens[w.N][:w.levels], arrival=t,
                                keep_result=False))
        srv.completed.clear()
        srv.failed.clear()
        srv.batches = 0
        made1 = srv.residents_made
        elapsed, done = run_stream(srv, reqs)
        st = latency_stats(done)
        results.append({"rate": rate, "requests": count, "completed": len(done),
                        "failed": len(srv.failed), "solves_per_s": len(done) / elapsed,
                        "batches": srv.batches, "peak_bytes": srv.peak_used,
                        "residents_made_while_serving": srv.residents_made - made1, **st})
    srv.close()
    torch.cuda.empty_cache()
    print(json.dumps({"mode": "serve", "metric": "served solves/s and latency (arrival -> host potentials)",
                      "unit": "solves/s", "budget_bytes": budget, "precision": "fp32",
                      "requests": "N in {32,64,128,256}, 3-10 levels, Poisson arrivals",
                      "density": "one seeded 1-4 Plummer density per N, sliced to the level count",
                      "residents_prewarmed": made0,
                      "device_bound": {"mix_solve_ms": mix_solve, "mix_solve_rate": 1e3 / mix_solve,
                                       "mix_with_copies_ms": mix_copies, "mix_with_copies_rate": 1e3 / mix_copies,
                                       "what": "mean over the 32 request shapes (uniform N and L) of one solve "
                                               "alone and of one solve with its upload and download, one at a "
                                               "time on one stream"},
                      "per_shape": per_shape,
                      "rates": results}))


# ----------------------------------------------------------------------------- table mode
def table_mode(args):
    """The baseline table: configs 1-4 on the GPU (FP64 plain, FP32, the cuFFT
    level convolutions) and through the FP64 oracle on the host (one core,
    and the level convolutions spread over all cores)."""
    import torch
    from paper_2301_06763_gb300 import build
    build.build()
    from paper_2301_06763_gb300 import nm, workloads as wl
    dev = torch.device("cuda", 0)

    def gpu_ms(w, rho, prec, method="original", reps=20):
        dt = torch.float32 if prec == "fp32" else torch.float64
        r = [torch.from_numpy(rho).to(dev, dt) for _ in range(2)]
        f = [torch.empty(rho.shape, dtype=torch.float64, device=dev) for _ in range(2)]
        with nm.Plan(w.levels, w.N, w.dx0, precision=prec, method=method) as p:
            for i in range(5):
                p.potential(r[i % 2], f[i % 2])
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for i in range(reps):
                p.potential(r[i % 2], f[i % 2])
            b.record()
            torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def cufft_ms(w, rho, prec, reps=10):
        dt = torch.float32 if prec == "fp32" else torch.float64
        with nm.Plan(w.levels, w.N, w.dx0) as p:
            sh = cufft_half_spectrum(torch, p.green_octant(), dev, dt)
        m = torch.from_numpy(np.concatenate([rho, rho[:-1]], axis=0)).to(dev, dt)   # 2L-1 fields
        for _ in range(3):
            cufft_level_convolutions(torch, m, sh)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            cufft_level_convolutions(torch, m, sh)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    workers = min(os.cpu_count() or 1, 16)
    pool = oracle_pool(workers)
    rows = []
    try:
        for name, w in (("1: 2x16^3", wl.config_small()), ("2: 4x64^3", wl.config_binary()),
                        ("3: 6x128^3", wl.config_contrast())):
            rho = w.rho()
            row = {"config": name, "gpu_fp64_ms": gpu_ms(w, rho, "fp64", reps=5 if w.N >= 128 else 20),
                   "gpu_fp32_ms": gpu_ms(w, rho, "fp32"), "cufft_fp32_ms": cufft_ms(w, rho, "fp32"),
                   "cufft_fp64_ms": cufft_ms(w, rho, "fp64", reps=3)}
            if w.levels == 4:
                row["gpu_fp64_dipole_ms"] = gpu_ms(w, rho, "fp64", "dipole")
                row["gpu_fp32_dipole_ms"] = gpu_ms(w, rho, "fp32", "dipole")
            _, t1 = oracle_solve_timed(rho, w.N, w.dx0, None)
            _, ta = oracle_solve_timed(rho, w.N, w.dx0, pool)
            row["oracle_1core_ms"] = t1 * 1e3
            row["oracle_all_cores_ms"] = ta * 1e3
            rows.append(row)
        meshes = wl.config_batch(seed=0)
        plans = [nm.Plan(w.levels, w.N, w.dx0, precision="fp32") for w in meshes]
        rhos = [w.rho() for w in meshes]
        r32 = [torch.from_numpy(r).to(dev, torch.float32) for r in rhos]
        phis = [torch.empty(r.shape, dtype=torch.float64, device=dev) for r in rhos]
        for _ in range(3):
            nm.batch_potential(plans, r32, phis)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(10):
            nm.batch_potential(plans, r32, phis)
        b.record()
        torch.cuda.synchronize()
        batch_ms = a.elapsed_time(b) / 10
        for p in plans:
            p.close()
        fp64_ms = sum(gpu_ms(w, r, "fp64", reps=2) for w, r in zip(meshes, rhos))
        cuf = sum(cufft_ms(w, r, "fp32", reps=2) for w, r in zip(meshes, rhos))
        sub = list(range(0, len(meshes), 8))          # every 8th mesh: 8 of 64
        t1 = sum(oracle_solve_timed(rhos[i], meshes[i].N, meshes[i].dx0, None)[1] for i in sub)
        ta = sum(oracle_solve_timed(rhos[i], meshes[i].N, meshes[i].dx0, pool)[1] for i in sub)
        scale = len(meshes) / len(sub)
        # the paper's runtime setting (Sect. 6 / Sect. 6's GPU runs): the oblate
        # ellipsoid on 8 levels of 128^3, timing only
        w = wl.config_paper_ellipsoid(N=128, levels=8)
        rho = w.rho()
        paper_row = {"config": "paper setting: ellipsoid 8x128^3", "gpu_fp64_ms": gpu_ms(w, rho, "fp64", reps=5),
                     "gpu_fp32_ms": gpu_ms(w, rho, "fp32"), "cufft_fp32_ms": cufft_ms(w, rho, "fp32"),
                     "cufft_fp64_ms": cufft_ms(w, rho, "fp64", reps=3)}
        _, ta = oracle_solve_timed(rho, w.N, w.dx0, pool)
        paper_row["oracle_all_cores_ms"] = ta * 1e3
        rows.append({"config": "4: batch of 64", "gpu_fp32_ms": batch_ms, "gpu_fp64_ms": fp64_ms,
                     "cufft_fp32_ms": cuf, "oracle_1core_ms": t1 * scale * 1e3,
                     "oracle_all_cores_ms": ta * scale * 1e3,
                     "note": "GPU FP32 = one nm_batch_potential; FP64 and cuFFT = the 64 meshes one by one; "
                             "oracle on 8 of the 64 meshes, scaled by 8"})
        # serving requests: the oracle on a sample of the stream's small meshes
        rng = np.random.default_rng(0)
        sample, t1 = [], 0.0
        for i in range(8):
            N = int(rng.choice([32, 64]))
            L = int(rng.integers(3, 11))
            ws = wl.Workload("serve-%d" % N, L, N, 1.0 / N, wl.random_plummers(rng, L, N))
            r = ws.rho()
            t1 += oracle_solve_timed(r, N, ws.dx0, pool)[1]
            sample.append("%dx%d" % (L, N))
        rows.append({"config": "5: serving requests (sample)", "oracle_all_cores_ms_per_request": t1 / 8 * 1e3,
                     "sample": sample, "note": "8 requests with N in {32, 64} from the request distribution"})
        rows.append(paper_row)
    finally:
        pool.shutdown()
    print(json.dumps({"mode": "table", "host_cores": os.cpu_count(), "oracle_workers": workers,
                      "cpu": platform.processor() or platform.machine(),
                      "cufft": "2L-1 level convolutions only (pad, R2C, multiply, C2R, crop) via torch.fft",
                      "rows": rows}))


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    elif args.mode == "batch":
        batch_mode(args)
    elif args.mode == "serve":
        serve_mode(args)
    elif args.mode == "accel":
        accel_mode(args)
    elif args.mode == "table":
        table_mode(args)
    elif args.mode == "fp32":
        fp32_mode(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
