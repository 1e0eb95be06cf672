"""The work items of the exact count with Lemma 2.3 (reversal, on top of
Lemma 2.2): the canonical enumeration of csrc/sk_mirror.cuh, compiled for the
host (tests/native/mirror_enum_check.cu, no GPU), must cover every orbit of
mirror-image items with total weight equal to the orbit's size, and the
mirrored walk must be closed under the mirror."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_mirror_item_enumeration_on_the_host():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "mirror_enum_check")
        subprocess.run([nvcc, "-std=c++17", "-O2", "-I",
                        os.path.join(ROOT, "paper_1507_00315_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "native", "mirror_enum_check.cu"), "-o", exe],
                       check=True, capture_output=True)
        r = subprocess.run([exe], capture_output=True, text=True)
    lines = r.stdout.strip().splitlines()
    assert lines[-1] == "total bad=0", "\n".join(l for l in lines if not l.endswith("bad=0"))
    assert r.returncode == 0
    assert len(lines) == sum(n - 1 for n in range(2, 13)) + 1
