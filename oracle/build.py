"""Build the CPU oracle (test infrastructure only).

libcloak_oracle.so: the FP64 oracle and the surrogate's CPU reference.  Plain gcc, no tuning flags:
-O2, no fast-math, no FMA contraction, OpenMP for the per-ray loops.

build_ext(kind): the same cloak_oracle.c in extended precision -- kind "ld" (long double: 64-bit
significand on x86-64, IEEE binary128 on AArch64), "q" (_Float128, IEEE binary128), "q_s64" (_Float128
with every state and stage point rounded to FP64) or "ld_f32" (long double with FP32 right-hand sides and
stage velocities outside the band r < R1 + 0.02) -- into libcloak_oracle_<kind>.so, for the rays FP64 or
FP32 cannot determine.  Built on demand only.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, f) for f in ("cloak_oracle.c", "surrogate_oracle.c")]
HDRS = [os.path.join(HERE, f) for f in ("cloak_oracle.h", "surrogate_oracle.h")]
LIB = os.path.join(HERE, "libcloak_oracle.so")
# q_s64: _Float128 with FP64 states; ld_f32: long double with FP32 right-hand sides outside the band near R1
EXT_KINDS = {"ld": 1, "q": 2, "q_s64": 2, "ld_f32": 1}
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
    defs = [f"-DORC_REAL_KIND={EXT_KINDS[kind]}"] + (["-DORC_STATE_F64=1"] if kind.endswith("_s64") else []) + \
        (["-DORC_MIXED_F32=1"] if kind.endswith("_f32") else [])
    cmd = ["gcc", *FLAGS, *defs, "-Wl,-Bsymbolic", "-o", lib + ".tmp", src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    if "--ext" in sys.argv:
        for k in EXT_KINDS:
            print(build_ext(k, force="--force" in sys.argv))
