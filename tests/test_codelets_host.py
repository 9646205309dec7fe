"""Host test of the register DFT codelets (csrc/codelets.cuh): radix 2, 4,
8 and 16 in both directions against the DFT sum in long double, including
the FP64 16-point codelet whose twiddle products are folded into fused
multiply-adds, which is also compared with the plain 16-point codelet.
Compiled by nvcc as host code (the codelets are __host__ __device__) and
run on the CPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_codelets(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = tmp_path / "codelet_test"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-x", "cu", "-I",
                    os.path.join(ROOT, "paper_0803_2386_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "codelet_test.cu"), "-o", str(exe)],
                   check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "codelets ok" in r.stdout
