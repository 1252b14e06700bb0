"""Build the CUDA library ``libapr.so`` for sm_103a, in-tree, with nvcc.

The translation units compile in parallel; the refinement, index and
time-step-bin units are compiled with ``--fmad=false`` so their float64
geometry and integration (split placement, merge centre of mass, lattice
quantisation, kicks, bin decisions) round exactly as written.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libapr.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
UNITS = {
    "apr_api.cu": [],
    "apr_index.cu": ["--fmad=false"],
    "apr_sph.cu": [],
    "apr_refine.cu": ["--fmad=false"],
    "apr_noalloc.cu": [],
    "apr_adjoint.cu": [],
    "apr_relax.cu": [],
    "apr_bins.cu": ["--fmad=false"],
    "apr_probe.cu": [],
}


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(INCLUDE, "apr.h"))
    return deps


def stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in _sources())


def build(force=False, verbose=False):
    """Compile and link ``libapr.so`` if any source is newer; return its path."""
    if not force and not stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    common = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
              "-Xptxas", "-v" if verbose else "-O3"]

    def one(unit):
        obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
        cmd = [cc, *common, *UNITS[unit], "-c", os.path.join(CSRC, unit), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {unit}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(len(UNITS)) as ex:
        results = list(ex.map(one, UNITS))
    if verbose:
        for _, err in results:
            print(err)
    tmp = LIB + ".tmp"
    cmd = [cc, ARCH, "-shared", "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
