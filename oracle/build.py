"""Compile the FP64 CPU oracle (oracle.c) into oracle/liboracle.so.

Test infrastructure: the library this builds is loaded only by the tests, the
smoke check and the CPU-baseline leg of the benchmark.  Strict IEEE build:
-O2 -ffp-contract=off, no fast-math, no -march=native.  OpenMP is used when the
compiler has it (the per-target / per-group loops are independent, and each
target's sum keeps its sequential order, so results do not depend on the
thread count).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-std=c99", "-Wall", SRC, "-o", tmp, "-lm"]
    for extra in (["-fopenmp"], []):
        r = subprocess.run(base[:1] + extra + base[1:], capture_output=True, text=True)
        if r.returncode == 0:
            break
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stderr)
    if verbose and r.stderr:
        print(r.stderr, file=sys.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
