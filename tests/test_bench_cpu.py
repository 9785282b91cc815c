"""bench.py's reference arm (the CPU oracle timed on the host cores) keeps the JSON contract on
CPU: one line with the arm's metric, a finite value, the per-step time actually measured, the
cpu_baseline and e2e objects, for a single step and without warm-up (small workload: the
216-atom cell's dense oracle solve)."""
import json
import math
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args, launcher=()):
    out = subprocess.run([sys.executable, *launcher, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run("--impl", "reference", "--workload", "1", "--steps", "1", "--warmup", "0")
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert math.isfinite(d["value"]) and d["value"] > 0
    assert d["ms_per_step"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["atoms"] == 216


def test_reference_arm_under_the_launcher_prints_one_line_from_rank_0():
    """Launched as two ranks by torch.distributed.run, rank 0 alone times the oracle and prints the line; the
    other rank exits 0 without work."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    launcher = ("-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                "--master-port", str(port))
    d = _run("--impl", "reference", "--gpus", "2", "--workload", "1", "--steps", "1", "--warmup", "0",
             launcher=launcher)
    assert d["impl"] == "reference" and math.isfinite(d["value"]) and d["value"] > 0

