"""Compile the CPU oracle (plain C, FP64) into oracle/liboracle.so.

The oracle is test infrastructure: tests, the smoke check and the benchmark's
CPU-baseline leg load it; the CUDA product path never does.  ``-ffp-contract=off``
keeps the compiler from fusing multiply-adds that the FP32 sampler
specification leaves unfused; OpenMP parallelises over samples.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "npp_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
