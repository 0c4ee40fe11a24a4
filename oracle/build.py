"""Build the FP64 CPU oracle (test infrastructure) into oracle/librise_oracle.so.

Plain gcc, no fast-math and no FMA contraction, so x86-64 and aarch64 hosts
produce the same doubles.  OpenMP is used when the compiler has it (the
parallel loops give the same results as one thread); without it the library
is built single-threaded.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rise_oracle.c")
LIB = os.path.join(HERE, "librise_oracle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    r = subprocess.run(base + ["-fopenmp", "-o", tmp, SRC, "-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base + ["-o", tmp, SRC, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
