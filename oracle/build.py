"""Build the FP64 CPU oracle (test infrastructure only) with gcc + OpenMP.

Plain portable C: no architecture flags, so it builds the same way on x86-64
and on aarch64 hosts.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bem_oracle.c")
SOURCES = (SRC, os.path.join(HERE, "bem_oracle_grad.c"))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libbem_oracle.so")


def stale() -> bool:
    """True when the library is missing or older than one of its sources."""
    if not os.path.exists(LIB):
        return True
    return os.path.getmtime(LIB) < max(os.path.getmtime(f) for f in SOURCES)


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and not stale():
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math", *SOURCES, "-o", LIB + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
