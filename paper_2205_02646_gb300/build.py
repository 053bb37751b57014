"""Build the sm_103a shared library ``librljsde.so`` in-tree with nvcc.

One nvcc invocation compiles the two translation units (CUDA kernels and the
host plan builder) in parallel for ``sm_103a`` only.
"""
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRC = [os.path.join(PKG, "csrc", "kernels.cu"), os.path.join(PKG, "csrc", "proposal.cu"),
       os.path.join(PKG, "csrc", "peak.cu"), os.path.join(PKG, "csrc", "plan.cpp")]
DEPS = SRC + [os.path.join(PKG, "csrc", "rljsde_internal.h"), os.path.join(ROOT, "include", "rljsde.h")]
LIB = os.path.join(PKG, "librljsde.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(d) for d in DEPS):
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "--threads", "4", "-shared",
           "-Xcompiler", "-fPIC,-fopenmp,-ffp-contract=off", "-I", os.path.join(ROOT, "include"),
           "-o", tmp] + SRC + ["-lgomp"]
    if verbose:
        cmd.insert(4, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
