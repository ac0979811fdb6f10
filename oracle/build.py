"""Compile the CPU oracle (lnr_oracle.c) into a shared library next to this file.

Test infrastructure: only tests, the smoke check and the benchmark's CPU baseline use
the result.  Flags: -O2 -ffp-contract=off (no implicit fused multiply-add, so the
oracle's FP32 steps are rounded exactly as written), no fast-math, OpenMP for the FP64
U-Net when the compiler supports it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lnr_oracle.c")
LIB = os.path.join(HERE, "liblnr_oracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            SRC, "-o", LIB + ".tmp", "-lm"]
    for extra in (["-fopenmp"], []):
        r = subprocess.run(base[:1] + extra + base[1:], capture_output=True, text=True)
        if r.returncode == 0:
            break
        if verbose:
            print(r.stderr, file=sys.stderr)
    else:
        raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
