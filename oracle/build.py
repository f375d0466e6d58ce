"""Compile the FP64 oracle (test infrastructure) into oracle/_build/liboracle.so.

Plain g++ -O3 with OpenMP, no architecture-specific flags and no floating-point
contraction or fast-math, so the same source gives the same results on x86-64
and aarch64 hosts and for any thread count.  Without OpenMP support in the
compiler the oracle is built single-threaded (same results, slower).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
SRC = os.path.join(HERE, "gs_oracle.cpp")


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "gs_oracle.h"))):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O3", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
           "-o", tmp, SRC]
    if subprocess.call(cmd) != 0:
        sys.stderr.write("oracle: building without OpenMP (single-threaded)\n")
        subprocess.check_call([c for c in cmd if c != "-fopenmp"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
