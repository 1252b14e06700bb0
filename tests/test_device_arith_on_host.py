"""Device arithmetic of the FP32-mixed step checked on the host.  Three header-only
pieces of the kernels are compiled for the CPU with nvcc and exercised against the
float64 operations they stand in for, on millions of values and the special ones:

* ``threshold_bits.cu``: apr_internal.cuh's list threshold ceil((2 h / delta)^2),
  read off the bits of the double with integer operations, against ceil() and the
  float64 conversion, with the integer root the threshold kernel derives from it
  (Sec. 2.3's neighbour criterion r < 2h on the integer lattice needs both exactly);
* ``dtmin_check.cu``: apr_dtmin.cuh's running minimum of the time-step criteria
  (Sec. 2.5), whose log-domain integer pre-test must leave the winners of the plain
  float64 cross products unchanged bit for bit, and the high-word bound it rests on;
* ``sinkpre_check.cu``: apr_sinkpre.cuh's float pre-test of the accretion radius
  (Sec. 3), which may reject only particles the float64 test rejects.

Each program exits 0 when every case agrees; a margin or guard made too small in
any of the headers makes it fail (checked by editing copies of the headers)."""
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


@pytest.mark.parametrize("program", ["threshold_bits.cu", "dtmin_check.cu", "sinkpre_check.cu"])
def test_device_arithmetic_on_host(program, tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / program.replace(".cu", ""))
    subprocess.run([nvcc, "-gencode=arch=compute_103a,code=sm_103a", "-std=c++17", "-O2",
                    "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2409_11470_gb300", "csrc"),
                    os.path.join(HERE, program), "-o", exe],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
