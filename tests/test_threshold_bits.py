"""The list thresholds' integer arithmetic on the host: apr_internal.cuh's
ceil((2 h / delta)^2), read off the bits of the double with integer operations, is
compiled for the CPU with nvcc (``threshold_bits.cu``) and compared with ceil() and
the float64 conversion on four million values and special ones, together with the
integer root the threshold kernel derives from it (Sec. 2.3's neighbour criterion
r < 2h on the integer lattice needs both exactly)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_threshold_bits_match_ceil(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "threshold_bits")
    subprocess.run([nvcc, "-gencode=arch=compute_103a,code=sm_103a", "-std=c++17", "-O2",
                    "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2409_11470_gb300", "csrc"),
                    os.path.join(HERE, "threshold_bits.cu"), "-o", exe],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 disagreements" in r.stdout
