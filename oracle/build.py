"""Build the CPU oracle's shared library (test infrastructure only).

g++ -O2 with -ffp-contract=off, so that every floating-point operation of the
oracle is a single IEEE-754 binary64 operation, rounded once, in source order.
OpenMP spreads the face and cell loops over the host cores; the arithmetic per
face and per cell is the same for any thread count.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liborc.so")
SRC = [os.path.join(HERE, "fv_oracle.cpp")]
DEPS = SRC + [os.path.join(HERE, "fv_oracle.hpp")]


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in DEPS):
            return LIB
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-Wall", "-o", LIB + ".tmp"] + SRC
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
