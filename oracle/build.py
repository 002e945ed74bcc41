"""Compile the C oracle into ``oracle/_build/liboracle.so`` (serial, the
reference the tests use) and ``oracle/_build/liboracle_omp.so`` (the same
source with OpenMP, a timing baseline on all host cores).

Test infrastructure only.  Plain gcc, no architecture-specific flags, so the
same source builds on the x86 development host and on the Arm GPU host.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
OMP_LIB_PATH = os.path.join(BUILD_DIR, "liboracle_omp.so")
SOURCES = [os.path.join(HERE, "pf_oracle.c")]
CFLAGS = ["-std=c11", "-O3", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off", "-Wno-unknown-pragmas"]


def flags(openmp: bool = False):
    """The gcc flags of a build (reported with the CPU baseline timings)."""
    return CFLAGS + (["-fopenmp"] if openmp else [])


def build(force: bool = False, openmp: bool = False) -> str:
    os.makedirs(BUILD_DIR, exist_ok=True)
    path = OMP_LIB_PATH if openmp else LIB_PATH
    newest = max(os.path.getmtime(p) for p in SOURCES + [os.path.join(HERE, "pf_oracle.h"), __file__])
    if not force and os.path.exists(path) and os.path.getmtime(path) >= newest:
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc"] + flags(openmp) + ["-o", tmp] + SOURCES + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


if __name__ == "__main__":
    print(build(force=True))
    print(build(force=True, openmp=True))
