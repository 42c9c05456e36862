"""Compile the oracle (plain C++17, FP64) into an in-tree shared library.

Test infrastructure only: the tests, the smoke check and the benchmark's
CPU-baseline leg load it.  No fused multiply-add contraction, no fast-math, so
every operation rounds as written.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["shower.cpp", "observables.cpp", "api.cpp"]
HEADERS = ["philox.hpp", "physics.hpp", "oracle_internal.hpp", "oracle_api.h"]
LIB = os.path.join(HERE, "_build", "liboracle.so")


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(os.path.join(HERE, f)) > t for f in SOURCES + HEADERS)


def build(force: bool = False) -> str:
    if force or needs_build():
        os.makedirs(os.path.dirname(LIB), exist_ok=True)
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-Wextra", "-o", tmp] + [os.path.join(HERE, s) for s in SOURCES]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
