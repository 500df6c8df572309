"""The integer-pipe FP64 product used by the wave kernels, checked on the CPU.

rs::dmul_int is plain integer arithmetic (__host__ __device__).  Compiled as
host code it must agree bit for bit with the CPU's IEEE multiply on every
input it does not flag as special: 60 million random operand pairs (random
bit patterns, rotation-like magnitudes, mantissas with long runs of ones and
zeros that produce exact ties) and a sweep of exponents near overflow and
underflow.  The GPU parity tests check the device build of the same code.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_dmul_int_matches_ieee_multiply(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "dmul_int_host")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_2412_01852_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), "-o", exe,
                    os.path.join(HERE, "native", "dmul_int_host.cu")], check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "bad=0" in r.stdout
