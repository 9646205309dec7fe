"""Host test of the per-device kernel set-up cache (csrc/device_once.h):
the set-up runs once per device ordinal, keeps each device's own value,
retries after a failure, refuses ordinals outside its table, and stays
consistent when many host threads launch at once.  Compiled with g++ and run
on the CPU; the same header guards every kernel launcher's attributes and
persistent grid sizes (running on two GPUs is not possible here)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_device_once(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "device_once_test"
    subprocess.run([gxx, "-std=c++17", "-O1", "-pthread", "-I",
                    os.path.join(ROOT, "paper_0803_2386_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "device_once_test.cpp"), "-o", str(exe)],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    assert "device_once ok" in r.stdout
