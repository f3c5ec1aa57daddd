"""Build the in-tree shared library libtc_b300.so (sm_103a) with nvcc.

Usage: python -m paper_2510_12011_b300.build   (or build() from Python).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libtc_b300.so")
SOURCES = ["mesh.cpp", "sim.cu", "mlp.cu"]
HEADERS = ["tc_internal.h", "kernels.cuh", "ionic_tp06.cuh", "exp2_table.inc", "mlp.cuh", "gemm_tc.cuh",
           "surrogate.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _newest_input():
    paths = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    paths.append(os.path.join(os.path.dirname(HERE), "include", "tc.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    nvcc = os.environ.get("NVCC", "nvcc")
    cmd = [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-shared",
           "-Xcompiler", "-fPIC,-fopenmp,-ffp-contract=off,-O3",
           "-Xptxas", "-v" if verbose else "-O3",
           "-o", LIB + ".tmp", *[os.path.join(CSRC, f) for f in SOURCES], "-lgomp"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + res.stdout + res.stderr)
    if verbose:
        sys.stderr.write(res.stdout + res.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
