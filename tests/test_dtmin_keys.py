"""The time-step limit's running minimum on the host: apr_dtmin.cuh compiled for the
CPU with nvcc (``dtmin_check.cu``).  Its log-domain integer pre-test may skip a
particle's float64 cross products only where they would not prefer it, so the
winners of add_keyed() and of the plain cross products (add()) agree bit for bit
over 200,000 sequences of random, near-tie and special values; and the bound the
pre-test rests on (the high word of a positive normal double within HL_ERR below
2^20 (log2 x + 1023)) holds on four million values, including the worst mantissa
1 / ln 2 (Sec. 2.5's Courant and force criteria)."""
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


def test_dtmin_keyed_winners_match_cross_products(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "dtmin_check")
    subprocess.run([nvcc, "-gencode=arch=compute_103a,code=sm_103a", "-std=c++17", "-O2",
                    "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2409_11470_gb300", "csrc"),
                    os.path.join(HERE, "dtmin_check.cu"), "-o", exe],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert " 0 disagreements" in r.stdout
