"""Build the CPU oracle (test infrastructure only).

libcloak_oracle.so: the FP64 oracle and the surrogate's CPU reference.  Plain gcc, no tuning flags:
-O2, no fast-math, no FMA contraction, OpenMP for the per-ray loops.

build_ext(kind): the same cloak_oracle.c in extended precision -- kind "ld" (long double: 64-bit
significand on x86-64, IEEE binary128 on AArch64) or "q" (_Float128, IEEE binary128) -- into
libcloak_oracle_<kind>.so, for the rays FP64 cannot determine.  Built on demand only.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, f) for f in ("cloak_oracle.c", "surrogate_oracle.c")]
HDRS = [os.path.join(HERE, f) for f in ("cloak_oracle.h", "surrogate_oracle.h")]
LIB = os.path.join(HERE, "libcloak_oracle.so")
EXT_KINDS = {"ld": 1, "q": 2}
FLAGS = ["-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-Wall"]


def _stale(lib, deps):
    return not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(f) for f in deps)


def build(force: bool = False) -> str:
    if not force and not _stale(LIB, SRCS + HDRS):
        return LIB
    cmd = ["gcc", *FLAGS, "-o", LIB + ".tmp", *SRCS, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


def ext_path(kind: str) -> str:
    return os.path.join(HERE, f"libcloak_oracle_{kind}.so")


def build_ext(kind: str = "ld", force: bool = False) -> str:
    if kind not in EXT_KINDS:
        raise ValueError(f"extended-precision kind must be one of {sorted(EXT_KINDS)}")
    lib = ext_path(kind)
    src = os.path.join(HERE, "cloak_oracle.c")
    if not force and not _stale(lib, [src, os.path.join(HERE, "cloak_oracle.h")]):
        return lib
    # -Bsymbolic: calls inside the library bind to its own (extended-precision) definitions
    cmd = ["gcc", *FLAGS, f"-DORC_REAL_KIND={EXT_KINDS[kind]}", "-Wl,-Bsymbolic", "-o", lib + ".tmp", src,
           "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    if "--ext" in sys.argv:
        for k in EXT_KINDS:
            print(build_ext(k, force="--force" in sys.argv))
