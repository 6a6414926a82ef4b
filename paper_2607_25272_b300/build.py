"""Build the SPCG CUDA library in-tree: paper_2607_25272_b300/libspcg.so.

nvcc compiles every translation unit of csrc/ for sm_103a (B300) and links
one shared library that exports the C ABI of include/spcg.h.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libspcg.so")
SOURCES = ["rng.cu", "fwht.cu", "qr.cu", "pcg.cu", "condest.cu", "api.cu", "noalloc.cu", "countsketch.cu", "mlp.cu", "batched.cu",
           "probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    raise RuntimeError("nvcc not found")


def build(verbose=False, ptxas_info=False):
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    newest = max(os.path.getmtime(p) for p in srcs + [os.path.join(CSRC, "common.cuh"),
                                                       os.path.join(CSRC, "internal.hpp"),
                                                       os.path.join(HERE, "..", "include", "spcg.h")])
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= newest and not ptxas_info:
        return LIB
    cmd = [nvcc(), "-O3", "-std=c++17", "-lineinfo", "-shared", "-Xcompiler", "-fPIC",
           "--expt-relaxed-constexpr", *ARCH, "-o", LIB, *srcs, "-lcudart"]
    if ptxas_info:
        cmd.insert(1, "-Xptxas=-v")
    if verbose:
        print(" ".join(cmd))
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("nvcc failed building libspcg.so")
    if ptxas_info:
        sys.stdout.write(res.stderr)
    return LIB


if __name__ == "__main__":
    build(verbose=True, ptxas_info="-v" in sys.argv)
    print(LIB)
