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

Under torchrun (N > 1) each rank solves its own copy of the workload (the
meshes are independent: replicas, weak scaling); the timed region is bracketed
by barriers and the maximum over ranks is reported.
"""
import argparse
import hashlib
import json
import os
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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--levels", type=int, default=6)
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle CPU timing (profiling runs)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--mode", choices=["solve", "batch", "serve"], default="solve")
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
def pass_bytes(name, N, fp32):
    """Algorithmic HBM bytes of one convolution pair in kernel `name` (level grid).

    The pass reads its input array once and writes its output once; the
    density and spectrum are read once.  Level grid: N^3 block, P = 2N."""
    es = 4 if fp32 else 8
    cs = 2 * es
    P = 2 * N
    n3 = N ** 3
    rows_in = N * N * P * cs           # [N][N][P] complex
    slab = N * P * P * cs              # [N][P][P] complex
    if name.startswith("xfwd"):
        return n3 * es + (N // 2) ** 3 * es + rows_in
    if name.startswith("yfwd"):
        return rows_in + slab
    if name.startswith("zseam"):
        return 2 * slab + (N + 1) ** 3 * es
    if name.startswith("yinv"):
        return slab + rows_in
    if name.startswith("xinv"):
        return rows_in + n3 * es + (N // 2 + 2) ** 3 * es
    return None


def source_hash():
    h = hashlib.sha256()
    for f in ("fft.cuh", "conv.cuh", "conv_inst.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2301_06763_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_name):
    """DRAM bytes per pair of `kernel_name` from the committed ncu summary, or
    None when no summary exists or the kernel sources changed since."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"source hash:\s*`?([0-9a-f]+)", text)
    if not m or m.group(1) != source_hash():
        return None
    m = re.search(r"^\|\s*%s\s*\|[^|]*\|[^|]*\|\s*([0-9.e+]+)\s*\|" % re.escape(kernel_name), text, re.M)
    return float(m.group(1)) if m else None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------- oracle timings
def cpu_baseline(levels, N):
    """The FP64 oracle, as it stands, on the host: one full convolution of a
    level (zero padding, 3-D transform, spectrum multiply, inverse, crop),
    extrapolated to the 2L - 1 convolutions of a solve."""
    import oracle
    from paper_2301_06763_gb300 import workloads as wl
    w = wl.config_contrast(levels=levels, N=N)
    rho = w.rho()
    spec = oracle.green_spectrum(N)
    t0 = time.perf_counter()
    oracle.isolated_convolution(rho[0] * w.dx0 ** 3, w.dx0, 1.0, spec)
    t = time.perf_counter() - t0
    nconv = 2 * levels - 1
    return {"value": 1.0 / (nconv * t), "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": "one oracle isolated_convolution of a %d^3 level (%.1f s), x%d "
                      "convolutions per solve; restriction/interpolation/assembly untimed"
                      % (N, t, nconv)}


def reference_arm(args):
    """--impl reference: the oracle on the host cores, bounded per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    N, L = args.N, args.levels
    P = 2 * N
    rng = np.random.default_rng(0)
    x = rng.standard_normal((P, P, P)) + 1j * rng.standard_normal((P, P, P))
    for _ in range(args.warmup):
        oracle.fft_axis(x, -1)
    times = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.fft_axis(x, -1)
        times.append(time.perf_counter() - t0)
    total = time.perf_counter() - t_all
    passes = 6 * (2 * L - 1)          # 3 forward + 3 inverse axis passes per convolution
    per_step = total / args.steps
    value = 1.0 / (passes * per_step)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "contrast-%dx%d" % (L, N), "levels": L, "N": N,
                   "precision": "fp64", "method": "original"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": "one oracle fft_axis pass over the (2N)^3 = %d^3 padded "
                                   "domain per step; a solve is %d such passes (%d convolutions"
                                   " x 6) plus untimed pad/multiply/crop/assembly" % (P, passes, 2 * L - 1)},
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
    """Pairwise dipole method (Sect. 7, Eqs. B.1-B.2) on 4 levels of 64^3 (two
    Plummer spheres), against the original method on the same mesh."""
    w = wl.config_binary()
    rho = w.rho()
    out = {"workload": "binary-4x64"}
    for prec, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
        r = torch.from_numpy(rho).to(dev, dt)
        phi = torch.empty(rho.shape, dtype=torch.float64, device=dev)
        for meth in ("original", "dipole"):
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
            out["%s_%s_ms" % (meth, prec)] = a.elapsed_time(b) / n
            p.close()
        out["overhead_%s" % prec] = out["dipole_%s_ms" % prec] / out["original_%s_ms" % prec]
    return out


def accel_rates(nm, torch, dev, rho, w, peak, reps=20):
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
    out = {"acceleration": {"workload": "contrast-%dx%d" % (L, N), "us_per_launch": us,
                            "algorithmic_bytes": 32 * cells, "gbs": gbs, "frac": gbs / peak}}
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
    out["interp_diagonal"] = diag
    return out


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
    clk = clocks.stop()

    # end to end through the host-buffer entry point (H2D + solve + D2H per step)
    h_rho = torch.from_numpy(rho.astype(np.float32)).pin_memory()
    h_phi = torch.empty(rho.shape, dtype=torch.float64).pin_memory()
    p32.potential_host(h_rho.numpy(), h_phi.numpy())
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        p32.potential_host(h_rho.numpy(), h_phi.numpy())
    e2e_s = max_over_ranks(torch, dist, time.perf_counter() - t0)

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
        bytes_launch = per_unit * du / dl
        achieved = bytes_launch / (dms / dl * 1e-3) / 1e9
        per_pair = ncu_traffic(dname)
        traffic = per_pair * du / dl if per_pair is not None else None
        roof = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "algorithmic_bytes_per_launch": bytes_launch,
                "avg_launch_ms": dms / dl}
    solve_bytes = sum(pass_bytes(k, N, True) * v[1] for k, v in stats.items()
                      if pass_bytes(k, N, True) is not None) / args.steps
    kernel_table = {k: {"launches": v[0], "avg_ms": v[2] / v[0], "share": v[2] / sum(
        x[2] for x in stats.values())} for k, v in sorted(stats.items(), key=lambda kv: -kv[1][2])}
    dip = dipole_rates(nm, wl, torch, dev) if not args.no_cpu_baseline else None
    ext = accel_rates(nm, torch, dev, rho, w, peak) if not args.no_cpu_baseline else {}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(L, N)
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "contrast-%dx%d" % (L, N), "levels": L, "N": N,
                   "precision": "fp32 passes, fp64 spectrum and final sum", "method": "original",
                   "l2": "%d rotating rho/phi sets (%.0f MB > L2)" % (
                       NSETS, NSETS * (rho.size * 4 + rho.size * 8) / 1e6),
                   "parallelism": "replicas" if world > 1 else "single",
                   "schedule": sched},
        "p50_ms": pct(per32, 50), "p99_ms": pct(per32, 99),
        "fp64": {"value": world * args.steps / (dev64_ms / 1e3), "unit": "solves/s",
                 "ms_per_step": dev64_ms / args.steps, "p50_ms": pct(per64, 50),
                 "p99_ms": pct(per64, 99), "dtype": "f64"},
        "hbm": {"solve_algorithmic_bytes": solve_bytes,
                "solve_gbs": solve_bytes / (ms_step * 1e-3) / 1e9,
                "frac": solve_bytes / (ms_step * 1e-3) / 1e9 / peak},
        "e2e": {"value": world * args.steps / e2e_s, "unit": "solves/s",
                "h2d_bytes_per_step": int(rho.size * 4), "d2h_bytes_per_step": int(rho.size * 8)},
        "gpu_launches": int(launches),
        "roofline": roof,
        "kernels": kernel_table,
        "cpu_baseline": cpu,
        "dipole": dip,
        "acceleration": ext.get("acceleration"),
        "interp_diagonal": ext.get("interp_diagonal"),
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
    ms_seq64 = timed(lambda: [p.potential(r, f) for p, r, f in zip(plans64, r64, phis)],
                     max(1, args.steps // 4))
    line = {"mode": "batch", "metric": "meshes/s, 64-mesh batch (N in {32,64,128}, 2-8 levels)",
            "unit": "meshes/s", "value": 64 / (ms_batch / 1e3), "ms_per_batch": ms_batch,
            "fp32_one_by_one_ms": ms_seq32, "fp64_plain_one_by_one_ms": ms_seq64,
            "speedup_vs_fp64_plain": ms_seq64 / ms_batch, "speedup_vs_fp32_one_by_one": ms_seq32 / ms_batch,
            "cells": cells, "kernels_per_batch_eager": per_batch_launches,
            "graph": "batch replayed as one CUDA graph after the first repeat",
            "shapes": sorted(set((w.levels, w.N) for w in meshes)),
            "schedules": {"%dx%d" % k: v for k, v in tuned.items()}, "steps": args.steps,
            "data": "synthetic", "dtype": "f32"}
    print(json.dumps(line))


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
    results = []
    for rate in [float(x) for x in args.rates.split(",")]:
        count = int(min(2000, max(20, rate * args.serve_seconds)))
        arrivals = wl.config_serving(rate, count=count, seed=0)
        reqs = []
        for i, (t, w) in enumerate(arrivals):
            reqs.append(Request(i, w.levels, w.N, w.dx0, dens[w.N][:w.levels], arrival=t,
                                keep_result=False))
        srv = Server(budget, slots=4, precision="fp32")
        # warm the pool: one request per shape, untimed
        warm = [Request(-1 - i, L, N, 1.0 / N, dens[N][:L], keep_result=False)
                for i, (L, N) in enumerate(sorted(set((r.levels, r.N) for r in reqs)))]
        run_stream(srv, warm)
        srv.completed.clear()
        elapsed, done = run_stream(srv, reqs)
        st = latency_stats(done)
        results.append({"rate": rate, "requests": count, "completed": len(done),
                        "failed": len(srv.failed), "solves_per_s": len(done) / elapsed,
                        "batches": srv.batches, "peak_bytes": srv.peak_used, **st})
        srv.close()
        torch.cuda.empty_cache()
    print(json.dumps({"mode": "serve", "metric": "served solves/s and latency (arrival -> host potentials)",
                      "unit": "solves/s", "budget_bytes": budget, "precision": "fp32",
                      "requests": "N in {32,64,128,256}, 3-10 levels, Poisson arrivals",
                      "density": "one seeded 1-4 Plummer density per N, sliced to the level count",
                      "rates": results}))


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    elif args.mode == "batch":
        batch_mode(args)
    elif args.mode == "serve":
        serve_mode(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
