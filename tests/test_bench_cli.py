"""bench.py's contract on the CPU: the module imports, every mode's entry
point exists, and the reference arm (the oracle on the host) prints one JSON
line with the keys the driver reads."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_entry_points_exist():
    for name in ("ours", "batch_mode", "serve_mode", "accel_mode", "table_mode", "reference_arm",
                 "cpu_baseline", "accel_rates", "dipole_rates", "cufft_baseline", "cufft_level_convolutions",
                 "oracle_solve_timed", "oracle_pool"):
        assert callable(getattr(bench, name)), name


def test_reference_arm_prints_one_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                          "--levels", "2", "--N", "16"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "solves/s" and d["value"] > 0
    for k in ("metric", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_oracle_solve_timed_matches_oracle():
    import numpy as np
    import oracle
    from paper_2301_06763_gb300 import workloads as wl
    w = wl.config_small()
    rho = w.rho()
    phi, t = bench.oracle_solve_timed(rho, w.N, w.dx0)
    assert t > 0
    assert np.max(np.abs(phi - oracle.solve(rho, w.N, w.dx0))) == 0.0


def test_traffic_summary_follows_the_kernel_sources(tmp_path, monkeypatch):
    # a traffic summary stamped with the current source hash is read back; a
    # comment or white-space edit keeps the hash, a code edit changes it and
    # the lookup then reports no traffic
    import shutil
    csrc = tmp_path / "paper_2301_06763_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.HASHED_SOURCES:
        shutil.copy(os.path.join(ROOT, "paper_2301_06763_gb300", "csrc", f), csrc / f)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    base = bench.source_hash()
    (tmp_path / "profiles" / "ncu_traffic.md").write_text(
        "source hash: `%s`\n\n| kernel | pairs | bytes per launch | c |\n|---|---|---|---|\n"
        "| zseam_f32_P256 | 6 | 7.5e8 | y |\n" % base)
    assert bench.ncu_traffic("zseam_f32_P256") == (6, 7.5e8)
    conv = csrc / "conv.cuh"
    conv.write_text("// a new comment\n" + conv.read_text().replace("namespace nm {", "namespace nm {\n\n/* block */ ", 1))
    assert bench.source_hash() == base
    assert bench.ncu_traffic("zseam_f32_P256") == (6, 7.5e8)
    conv.write_text(conv.read_text().replace("constexpr int kMaxPairs = 64;", "constexpr int kMaxPairs = 65;"))
    assert bench.source_hash() != base
    assert bench.ncu_traffic("zseam_f32_P256") is None


def test_launch_bytes_count_one_half_pair_per_solve():
    # the finest pair of an original-method solve needs only kx <= N
    N = 128
    full = bench.pass_bytes("zseam_f32_P256", N, True)
    half = bench.pass_bytes("zseam_f32_P256", N, True, half=True)
    assert half < full and abs(half - (2 * N * 2 * N * (N + 1) * 8 + (N + 1) ** 3 * 4)) == 0
    assert bench.launch_bytes("zseam_f32_P256", N, True, 6, 1) == 5 * full + half
    assert bench.launch_bytes("restrict_f32", N, True, 5, 5) is None
