"""Compile the oracle's C source into ``oracle/liboracle.so`` with gcc (plain -O2, no
vector intrinsics and no -march flags, so it builds the same on x86_64 and aarch64).

OpenMP (-fopenmp) is used when the compiler supports it; the loops it shares among threads
compute the same results for any thread count (see oracle.c), and without it the library is
single-threaded."""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "oracle.c")
OUT = os.path.join(_HERE, "liboracle.so")
_BASE = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off"]


def build(force: bool = False) -> str:
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= os.path.getmtime(SRC):
        return OUT
    tmp = OUT + f".tmp{os.getpid()}"
    try:
        subprocess.check_call(_BASE + ["-fopenmp", "-o", tmp, SRC, "-lm"], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(_BASE + ["-o", tmp, SRC, "-lm"])
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True))
