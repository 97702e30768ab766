"""Compile the FP64 oracle into oracle/libgmr_oracle.so (test infrastructure).

Plain g++ with -ffp-contract=off and without -ffast-math, so that every
floating-point operation is a separately rounded IEEE-754 operation; the FP32
binning specification relies on that. -fopenmp for the loops over pixels,
records and faces (results do not depend on the thread count).
"""

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gmr_oracle.cpp")
LIB = os.path.join(HERE, "libgmr_oracle.so")
FLAGS = ["-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp"]


def build(force: bool = False) -> str:
    override = os.environ.get("GMR_ORACLE_LIB")
    if override:
        return override
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["g++", *FLAGS, "-Wall", "-o", LIB + ".tmp", SRC]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
