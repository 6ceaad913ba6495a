"""Compile the FP64 CPU oracle (sph_oracle.c) into oracle/liboracle.so.

Test infrastructure only: the oracle is built so that tests, the smoke check
and the benchmark's CPU-baseline leg can load it.  Plain gcc, no cmake.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sph_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Build liboracle.so if missing or older than its sources; return its path."""
    deps = [SRC, os.path.join(HERE, "sph_oracle.h")]
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in deps)):
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    compile_source(SRC, tmp)
    os.replace(tmp, LIB)
    return LIB


def compile_source(src: str, out: str) -> str:
    """Compile one oracle source (sph_oracle.c, or a test's patched copy of
    it) into the shared library `out`.  -ffp-contract=off: no fused
    multiply-add, so x86 and Arm hosts give the same FP64 rounding."""
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-Wall", "-I", HERE, "-o", out, src, "-lm"]
    subprocess.check_call(cmd)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
