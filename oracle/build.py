"""Build the FP64 CPU oracle (test infrastructure) into oracle/liboracle.so.

Plain g++ with OpenMP; no CUDA.  Called by the oracle wrapper on first import
and by the top-level build step.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.cpp")
SRCS = [SRC, os.path.join(HERE, "pchain.cpp")]
HDR = os.path.join(HERE, "oracle.h")
LIB = os.path.join(HERE, "liboracle.so")


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in SRCS + [HDR])


def build(force: bool = False) -> str:
    if force or needs_build():
        tmp = LIB + ".tmp.%d" % os.getpid()
        cmd = ["g++", "-std=c++17", "-O2", "-fcx-limited-range", "-fopenmp",
               "-fPIC", "-shared", "-Wall", "-o", tmp] + SRCS
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
