"""Builds libace.so in-tree: the CUDA decoder (sm_103a) and the host encoder.

nvcc -gencode arch=compute_103a,code=sm_103a compiles the device code; the
encoder is plain C++17 for the host.  Both objects compile in parallel and
link into one shared library with the shared CUDA runtime, so the process
shares one runtime with PyTorch.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libace.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["ace.cu", "encoder_gpu.cu"]
CPP_SOURCES = ["encoder.cpp"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA 13 toolkit is required to build libace.so")
    return cand


def _sources():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    out.append(os.path.abspath(__file__))
    return out


def needs_build():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _sources())


def build(force=False, verbose=False):
    """Compile and link libace.so if any source is newer; returns its path."""
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]
    jobs = []
    objs = []
    for f in CU_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append([nvcc] + ARCH + common + ["-lineinfo", "-Xptxas", "-v", "-c",
                                              os.path.join(CSRC, f), "-o", o])
    for f in CPP_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-I" + INCLUDE,
                     "-I/usr/local/cuda/include", "-c", os.path.join(CSRC, f), "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n%s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        return r.stdout + r.stderr

    with ThreadPoolExecutor(len(jobs)) as ex:
        logs = list(ex.map(run, jobs))
    if verbose:
        sys.stdout.write("".join(logs))
    with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
        f.write("".join(logs))
    tmp = LIB + ".%d.tmp" % os.getpid()
    run([nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + ["-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
