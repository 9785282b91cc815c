"""Plan tables that the matvec kernels index with (csrc/qeq_internal.cuh), checked on the host: nvcc
compiles tests/native/plan_tables_check.cu for the CPU (no GPU needed).  For every mesh length the plan
can choose (2^a 3^b 5^c up to 1024): the FFT radices (product K, fewest stages by brute force) and stage
constants of both radix limits, the frequency and position tables as inverse permutations, the
magic-number index division equal to n / d for every divisor the plans carry (exhaustive below 2^22),
and, for B-spline orders 4, 6 and 8, each spread brick's candidate bins against a brute-force search of
the stencil bases that reach it.  For a set of mesh shapes and line counts: every FFT line of the z, y
and inverse-y work lists covered once, every x line once as itself or as its mirror.  For pairs of fine
and coarse lengths: the preconditioner's coarse-spread tiles hold every stencil point of their atoms."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not available")
def test_plan_tables_on_the_host(tmp_path):
    exe = str(tmp_path / "plan_tables_check")
    subprocess.check_call(["nvcc", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-o", exe,
                           os.path.join(ROOT, "tests", "native", "plan_tables_check.cu")])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(out.stdout)
    assert out.returncode == 0, out.stdout + out.stderr
