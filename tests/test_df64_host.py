"""The double-float arithmetic of the df64 kernels, checked on the host.

csrc/df64.cuh's operations are __host__ __device__; tests/df64_host_check.cu
builds them as host code (nvcc, no GPU needed) and checks, against FP64 and
long-double references: TwoSum / TwoProd are error-free; df add, multiply and
fma (also with an FP32 operand) are accurate to 2^-44; the lazy product sums
of the sparse products to K * 2^-46 of the sum of magnitudes; the identity
block shortcut gives the same bits as the products it replaces; a double's
split into hi + lo keeps 48 bits.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_df64_arithmetic_on_host(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "df64_host_check")
    inc = os.path.join(os.path.dirname(HERE), "include")
    cmd = [nvcc, "-O2", "-std=c++17", "-Xcompiler", "-ffp-contract=off", f"-I{inc}",
           os.path.join(HERE, "df64_host_check.cu"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(out.stdout)
    assert out.returncode == 0 and out.stdout.strip().endswith("OK"), out.stdout + out.stderr
