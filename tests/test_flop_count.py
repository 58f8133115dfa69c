"""The per-pair arithmetic of the rooflines: C_tt, the flops of one
triangle-triangle distance, is counted on the oracle's own routine
(tests/flops/oracle_flops.cpp: oracle.c compiled with a counting number type),
and the kernels' routine is counted beside it (tests/flops/kernel_flops.cu:
the kernels' template instantiated on the host with the same counting type,
for the executed-work figures).  Both must be the numbers the benchmark uses.
Host code only, no GPU."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FLOPS = os.path.join(ROOT, "tests", "flops")


def _run(exe):
    mean, lo, hi = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return float(mean), int(lo), int(hi)


def test_oracle_tritri_flops_match_the_benchmark(tmp_path):
    exe = tmp_path / "oracle_flops"
    subprocess.run(["g++", "-O1", "-fopenmp", "-ffp-contract=off", "-o", str(exe),
                    os.path.join(FLOPS, "oracle_flops.cpp")], check=True, capture_output=True)
    mean, lo, hi = _run(exe)
    sys.path.insert(0, ROOT)
    import bench
    assert mean == bench.FLOPS_PER_PAIR
    assert lo <= mean <= hi


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_kernel_tritri_flops_match_the_benchmark(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / "kernel_flops"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    "-I", os.path.join(ROOT, "paper_1711_07663_gb300", "csrc"), "-o", str(exe),
                    os.path.join(FLOPS, "kernel_flops.cu")], check=True, capture_output=True)
    mean, lo, hi = _run(exe)
    sys.path.insert(0, ROOT)
    import bench
    assert mean == bench.FLOPS_PER_PAIR_KERNEL
    assert lo <= mean <= hi
