"""Builds liblbm.so (the C-ABI CUDA library) in-tree for sm_103a.

    python -m paper_2206_00946_gb300.build

One translation unit, nvcc, -gencode arch=compute_103a,code=sm_103a; the
CUDA runtime is linked statically so the library only needs the driver.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "_lib", "liblbm.so")
SOURCES = ["lbm_api.cu", "lbm_noalloc.cu", "lbm_adjoint.cu", "lbm_batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh"))]
    files.append(os.path.join(INCLUDE, "lbm.h"))
    return files


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build_lib(force: bool = False, verbose: bool = False, extra=(), out: str = None) -> str:
    LIB_ = out or LIB
    if not force and os.path.exists(LIB_) and os.path.getmtime(LIB_) >= max(os.path.getmtime(f) for f in _inputs()):
        return LIB_
    os.makedirs(os.path.dirname(LIB_), exist_ok=True)
    tmp = LIB_ + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-cudart", "static", "-I", INCLUDE, "-I", CSRC, *extra,
           "-o", tmp, *[os.path.join(CSRC, s) for s in SOURCES]]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_)
    return LIB_


if __name__ == "__main__":
    import argparse

    ap = argparse.ArgumentParser()
    ap.add_argument("-v", action="store_true")
    ap.add_argument("--ptxas", action="store_true")
    ap.add_argument("--out", default=None)
    ap.add_argument("-D", action="append", default=[], help="extra preprocessor definitions")
    a = ap.parse_args()
    extra = (["-Xptxas", "-v"] if a.ptxas else []) + [f"-D{d}" for d in a.D]
    print(build_lib(force=True, verbose=a.v, extra=extra, out=a.out))
