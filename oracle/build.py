"""Compile the FP64 CPU oracle into oracle/libmine_oracle.so.

Test infrastructure only: the product library never links or loads it.
Plain gcc, OpenMP over pairs, FP contraction off so that every expression in
the oracle rounds exactly as written (no fused multiply-add on either the
x86-64 host or the aarch64 GPU host).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mine_oracle.c")
LIB = os.path.join(HERE, "libmine_oracle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-Wall", "-Wextra",
           "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
