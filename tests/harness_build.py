"""Builds the host harnesses of the CPU tests (test infrastructure).

Each harness is compiled by nvcc for the host into tests/harness/_build/ (ignored by
git), under a name that encodes a hash of the harness, the library sources and the
flags, so that a test session reuses a build made from the same sources.
"""
import glob
import hashlib
import os
import shutil
import subprocess

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "harness")
ROOT = os.path.dirname(os.path.dirname(HERE))
CSRC = os.path.join(ROOT, "paper_2206_00946_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")


def nvcc():
    """Path of nvcc, or None when the CUDA toolkit is not installed."""
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand if os.path.exists(cand) else None


def build_harness(name, flags=()):
    """Compiles tests/harness/<name>.cu into a shared library and returns its path."""
    src = os.path.join(HERE, name + ".cu")
    h = hashlib.sha256(" ".join(flags).encode())
    for f in [src] + sorted(glob.glob(os.path.join(CSRC, "*.cu*"))) + [os.path.join(INCLUDE, "lbm.h")]:
        h.update(open(f, "rb").read())
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, f"{name}-{h.hexdigest()[:16]}.so")
    if not os.path.exists(so):
        tmp = f"{so}.tmp{os.getpid()}"
        subprocess.run([nvcc(), *flags, "-std=c++17", "-O2", "-shared", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                        "-I", CSRC, src, "-o", tmp], check=True)
        os.replace(tmp, so)
    return so
