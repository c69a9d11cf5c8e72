"""Builds the FP64 CPU oracle (``libfuncsne_oracle.so``) with gcc.

Test infrastructure only: the oracle is loaded by the test-suite, the smoke
check and the benchmark's CPU-baseline leg, never by the product path.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "funcsne_oracle.c")
LIB = os.path.join(HERE, "libfuncsne_oracle.so")


def build_oracle(force: bool = False) -> str:
    """Compile the oracle if the library is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    # OpenMP over points: results are identical for any thread count
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
