"""Double-float arithmetic of the final checks' FFT passes (csrc/dd.cuh), checked on the host:
nvcc compiles tests/native/dd_check.cu for the CPU (no GPU needed) and the program compares
conversion, sums, products and a 64-point DFT with FP64 against the bounds the kernels rely on
(2^-44 relative per operation; 1e-11 of the transform's size)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not available")
def test_double_float_arithmetic_bounds(tmp_path):
    exe = str(tmp_path / "dd_check")
    subprocess.check_call(["nvcc", "-O2", "-std=c++17", "-Xcompiler", "-ffp-contract=off", "-o", exe,
                           os.path.join(ROOT, "tests", "native", "dd_check.cu")])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    print(out.stdout)
    assert out.returncode == 0, out.stdout + out.stderr
