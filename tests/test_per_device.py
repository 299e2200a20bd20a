"""Per-device kernel set-up (shared-memory limits, occupancy) is kept per
device index, not once per process: the host-side bookkeeping, compiled with
the host compiler and run without a GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_per_device_bookkeeping(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "per_device_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", os.path.join(HERE, "native", "per_device_check.cpp"),
                    "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
