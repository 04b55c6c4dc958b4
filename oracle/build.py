"""Compile the FP64 oracle (plain C) into ``oracle/liboracle_das.so``.

The oracle is test infrastructure: this script only builds it.  Flags keep every
floating-point operation exactly as written (no contraction into fused multiply-add,
no fast-math), which the float32 "contract" delay mode relies on.  OpenMP is used if
the compiler supports it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "das_oracle.c")
LIB = os.path.join(HERE, "liboracle_das.so")


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    base = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", SRC, "-o", LIB + ".tmp"]
    for extra in (["-fopenmp"], []):
        r = subprocess.run(base[:1] + extra + base[1:] + ["-lm"], capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(LIB + ".tmp", LIB)
            if verbose:
                print("built", LIB, "with", extra or "no OpenMP")
            return LIB
    raise RuntimeError("oracle build failed:\n" + r.stderr)


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
