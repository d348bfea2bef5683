"""Build the FP64 CPU oracle (test infrastructure) into oracle/libkgoracle.so.

Plain gcc, IEEE double with no fused multiply-add contraction (-ffp-contract=off),
OpenMP over independent lines only.  Used by the test suite, the package smoke
check and the CPU-baseline leg of the benchmark; never by the GPU library.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kg_oracle.c")
LIB = os.path.join(HERE, "libkgoracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "kg_oracle.h"))
    ):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-Wall", "-Wextra", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
