"""In-tree build of libgks.so (CUDA kernels for sm_103a + host C++).

The translation units compile in parallel; objects go to ``_build/`` next to
this file and the shared library to ``libgks.so`` beside it.  Nothing is
installed anywhere else.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgks.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
# The reconstruction and flux kernels (and the one-launch stage that inlines
# them) take FP32 division and square root from the hardware approximations
# (within 2 ulp) and flush FP32 denormals: these flags touch single precision
# only, so the FP64 path is unchanged, and the FP32-bulk path stays inside its
# tolerance against the FP64 oracle.  The cell-update kernels keep IEEE FP32
# arithmetic.
FAST_FP32 = ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]
FAST_UNITS = ("gks_recon.cu", "gks_flux.cu", "gks_flux_xw.cu", "gks_stage.cu")


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgks")


def _sources():
    cu = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith(".cu")]
    cpp = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith(".cpp")]
    hdr = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hdr.append(os.path.join(INCLUDE, "gks.h"))
    return cu, cpp, hdr


def _compile(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed:\n%s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r.stderr


def build(force=False, verbose=False):
    """Compile libgks.so if any source is newer than it; return its path."""
    cu, cpp, hdr = _sources()
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(p) for p in cu + cpp + hdr + [__file__])
        if os.path.getmtime(LIB) >= newest:
            return LIB
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    jobs, objs = [], []
    for src in cu:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        jobs.append([nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17"] +
                    (FAST_FP32 if os.path.basename(src) in FAST_UNITS else []) +
                    ["-Xcompiler", "-fPIC",
                     "-Xcompiler", "-ffp-contract=off", "--expt-relaxed-constexpr",
                     "-I", INCLUDE, "-c", src, "-o", obj])
    for src in cpp:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall",
                     "-I", os.path.join(cuda, "include"), "-I", INCLUDE, "-c", src, "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        logs = list(ex.map(_compile, jobs))
    if verbose:
        for log in logs:
            if log:
                print(log)
    tmp = LIB + ".tmp%d" % os.getpid()
    _compile([nvcc, ARCH, "-shared", "-cudart=static", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
