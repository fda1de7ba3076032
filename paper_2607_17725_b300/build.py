"""Build the in-tree shared library libfastvem.so (host topology with g++,
CUDA kernels and the C ABI with nvcc for sm_103a)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libfastvem.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout)
        raise RuntimeError("build step failed: " + " ".join(cmd))
    return r.stdout


def sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))
            if f.endswith((".cpp", ".cu", ".h", ".cuh"))] + \
        [os.path.join(os.path.dirname(HERE), "include", "fastvem.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(force=False, verbose=False):
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    objs = []
    for f in ("topo.cpp", "plan.cpp"):
        o = os.path.join(OUT, f.replace(".cpp", ".o"))
        _run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-Wall", "-c",
              os.path.join(CSRC, f), "-o", o])
        objs.append(o)
    o = os.path.join(OUT, "fastvem.o")
    out = _run(["nvcc", "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
                "-Xptxas", "-v" if verbose else "-O3", "-c", os.path.join(CSRC, "fastvem.cu"), "-o", o])
    if verbose:
        sys.stdout.write(out)
    objs.append(o)
    tmp = LIB + ".tmp"
    _run(["nvcc", "-shared", *ARCH, "-Xcompiler", "-fopenmp", "-o", tmp, *objs, "-lgomp"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
