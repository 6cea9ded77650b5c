"""Compile the FP64 CPU oracle into oracle/liboracle_swe.so (test infrastructure).

Plain g++, -O2 with floating-point contraction off so every product and sum
rounds on its own, as the source is written; OpenMP for the optional
multi-threaded edge and cell loops (serial by default).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "swe_oracle.cpp")
LIB = os.path.join(HERE, "liboracle_swe.so")


def command() -> list[str]:
    return ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
            "-shared", SRC, "-o", LIB]


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    subprocess.run(command(), check=True)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv)
    print(LIB)
