"""FFT plan tables and the kernels' magic-number index division (csrc/qeq_internal.cuh), checked on
the host: nvcc compiles tests/native/fft_tables_check.cu for the CPU (no GPU needed) and the program
checks, for every mesh length the plan can choose (2^a 3^b 5^c up to 1024) and both radix limits,
the radices (product K, fewest stages by brute force), the stage constants, that the frequency and
position tables are inverse permutations, and that the division equals n / d for every divisor the
plans carry (exhaustive below 2^22)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not available")
def test_fft_plan_tables_and_index_division(tmp_path):
    exe = str(tmp_path / "fft_tables_check")
    subprocess.check_call(["nvcc", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-o", exe,
                           os.path.join(ROOT, "tests", "native", "fft_tables_check.cu")])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(out.stdout)
    assert out.returncode == 0, out.stdout + out.stderr
