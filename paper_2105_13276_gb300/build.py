"""Build ``libdmr.so`` in-tree with nvcc for sm_103a (GB300).

One translation unit, one -gencode, no cmake: a few seconds on x86 and on
the Arm GPU hosts.  ``-fmad=false``: nothing is contracted behind the
source's back; the fused multiply-adds of the FP64 update formulas are
written out in the kernels, the same in every code path.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "libdmr.so")

SOURCES = ["dmr.cu", "dmr_noalloc.cu"]
HEADERS = ["dmr_kernels.cuh", "dmr_adjoint.cuh", "dmr_period.cuh"]

ARCH = "-gencode=arch=compute_103a,code=sm_103a"
FLAGS = ["-O3", "-lineinfo", "-fmad=false", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
         "-shared", "--expt-relaxed-constexpr"]


def nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _stale():
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(INCLUDE, "dmr.h"),
                                                                 os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Compile libdmr.so unless it is up to date; returns its path."""
    if not force and not _stale():
        return OUT
    tmp = OUT + ".tmp%d" % os.getpid()
    cmd = [nvcc(), ARCH] + FLAGS + ["-I" + INCLUDE, "-o", tmp] + [os.path.join(CSRC, s) for s in SOURCES]
    if verbose:
        print(" ".join(cmd))
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True, verbose=True))
