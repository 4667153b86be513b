"""Build the CPU FP64 oracle (test infrastructure only) into oracle/libcloak_oracle.so.

Plain gcc, no tuning flags: -O2, no fast-math, no FMA contraction, OpenMP for
the per-ray loops.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, f) for f in ("cloak_oracle.c", "surrogate_oracle.c")]
HDRS = [os.path.join(HERE, f) for f in ("cloak_oracle.h", "surrogate_oracle.h")]
LIB = os.path.join(HERE, "libcloak_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(f) for f in SRCS + HDRS):
        return LIB
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-Wall", "-o", LIB + ".tmp", *SRCS, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
