"""The exact kernel's per-term digit product, on the host, for every (delta,
n) plan the library compiles (tests/native/digit_plan_check.cu, compiled
with nvcc for the host only; no GPU): the digits times the tail product
equal the exact product of the correlations, the digits below the top are
non-negative, and each plan's walk-width bound keeps its 64-bit item sums
exact."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_digit_plan_on_the_host():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "digit_plan_check")
        subprocess.run([nvcc, "-std=c++17", "-O2", "-I",
                        os.path.join(ROOT, "paper_1507_00315_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "native", "digit_plan_check.cu"), "-o", exe],
                       check=True, capture_output=True)
        r = subprocess.run([exe], capture_output=True, text=True)
    lines = r.stdout.strip().splitlines()
    assert lines[-1] == "total bad=0", "\n".join(l for l in lines if not l.endswith("bad=0"))
    assert r.returncode == 0
    assert len(lines) == 2 * 31 + 1
