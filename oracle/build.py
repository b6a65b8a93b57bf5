"""Builds the FP64 CPU oracle (test infrastructure) as oracle/liblbm_oracle.so.

Plain gcc, -O2, no -ffast-math and no -march flags, so that it gives the same
results on x86-64 and aarch64 hosts.  build_oracle(omp=True) builds the same
source with -fopenmp as oracle/liblbm_oracle_omp.so: its per-cell loops over z
run on all host cores with bit-identical results (the benchmark's all-core CPU
baseline).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
LIB = os.path.join(HERE, "liblbm_oracle.so")
LIB_OMP = os.path.join(HERE, "liblbm_oracle_omp.so")


def build_oracle(force: bool = False, omp: bool = False) -> str:
    lib = LIB_OMP if omp else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "lbm_oracle.h"))
    ):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-ffp-contract=off",
           *(["-fopenmp"] if omp else []), "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build_oracle(force=True))
    print(build_oracle(force=True, omp=True))
