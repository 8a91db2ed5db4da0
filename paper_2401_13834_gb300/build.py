"""Build the in-tree shared library libtransientx_gb300.so for sm_103a.

    python -m paper_2401_13834_gb300.build [--force]

Translation units: plan.cpp (host tables, g++ with -ffp-contract=off so the
Eq. 1 delay tables round identically on every host) and every .cu file under
csrc/ (nvcc, -gencode arch=compute_103a,code=sm_103a): kernels.cu (single
beam) and batch.cu (batched execute), both on the kernels in kernels.cuh.
They compile in parallel and link with nvcc -shared. The result lives next to this file under _lib/.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUTDIR = os.path.join(HERE, "_lib")
LIBNAME = "libtransientx_gb300.so"
LIBPATH = os.path.join(OUTDIR, LIBNAME)
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found (set NVCC or put the CUDA toolkit on PATH)")


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))
            if f.endswith((".cu", ".cpp", ".h", ".cuh"))] + [os.path.join(INCLUDE, "transientx.h")]


def _stale() -> bool:
    if not os.path.exists(LIBPATH):
        return True
    t = os.path.getmtime(LIBPATH)
    return any(os.path.getmtime(s) > t for s in _sources())


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the library if any source is newer than it; return its path."""
    if not force and not _stale():
        return LIBPATH
    os.makedirs(OUTDIR, exist_ok=True)
    nvcc = _nvcc()
    cxx = os.environ.get("CXX", "g++")
    objs, cmds = [], []
    obj_plan = os.path.join(OUTDIR, "plan.o")
    cmds.append([cxx, "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall", "-I", INCLUDE,
                 "-I", CSRC, "-c", os.path.join(CSRC, "plan.cpp"), "-o", obj_plan])
    objs.append(obj_plan)
    for cu in sorted(f for f in os.listdir(CSRC) if f.endswith(".cu")):
        obj = os.path.join(OUTDIR, cu[:-3] + ".o")
        cmds.append([nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
                     "-Xptxas", "-v" if verbose else "-O3",
                     "-I", INCLUDE, "-I", CSRC, "-c", os.path.join(CSRC, cu), "-o", obj])
        objs.append(obj)
    with ThreadPoolExecutor(len(cmds)) as ex:
        outs = list(ex.map(_run, cmds))
    if verbose:
        for o in outs:
            sys.stdout.write(o)
    tmp = LIBPATH + ".tmp"
    _run([nvcc, ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
    os.replace(tmp, LIBPATH)
    return LIBPATH


if __name__ == "__main__":
    p = build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(p)
