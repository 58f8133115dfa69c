"""The per-pair arithmetic the benchmark's rooflines use is the count the flop
counter (csrc/flopcount.cu: the kernels' triangle-pair routine instantiated
with a counting number type) reports; host code only, no GPU."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_flops_per_pair_matches_the_counter(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / "flopcount"
    src = os.path.join(ROOT, "paper_1711_07663_gb300", "csrc", "flopcount.cu")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-o", str(exe), src],
                   check=True, capture_output=True)
    mean, lo, hi = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    sys.path.insert(0, ROOT)
    import bench
    assert float(mean) == bench.FLOPS_PER_PAIR
    assert int(lo) <= float(mean) <= int(hi)
