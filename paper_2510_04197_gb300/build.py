"""Build libdvbm.so in-tree with nvcc for sm_103a (no cmake, no torch extension).

The translation units compile in parallel; the shared library lands next to
this file, with libdvbm_probe.so (the FP64 throughput probe bench.py uses).
Usage: ``python -m paper_2510_04197_gb300.build`` or ``build()``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libdvbm.so")
SOURCES = ["dvbm_step.cu", "dvbm_aux.cu", "dvbm_api.cu", "dvbm_noalloc.cu", "dvbm_adjoint.cu", "dvbm_d2q16.cu"]
# the FP64 throughput probe bench.py reports the step's FP64 work against
PROBE_SOURCE, PROBE_OUT = "dvbm_probe.cu", os.path.join(HERE, "libdvbm_probe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdvbm")
    return exe


def _compile(src: str, builddir: str, verbose: bool) -> str:
    obj = os.path.join(builddir, src.replace(".cu", ".o"))
    cmd = [nvcc(), *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        print(r.stderr)
    return obj


def build(verbose: bool = False) -> str:
    builddir = os.path.join(HERE, "_build")
    os.makedirs(builddir, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES) + 1) as ex:
        objs = list(ex.map(lambda s: _compile(s, builddir, verbose), SOURCES + [PROBE_SOURCE]))
    probe_obj = objs.pop()
    r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", PROBE_OUT + ".tmp", probe_obj, "-lcudart"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link of the probe failed:\n{r.stdout}\n{r.stderr}")
    os.replace(PROBE_OUT + ".tmp", PROBE_OUT)
    tmp = OUT + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv))
