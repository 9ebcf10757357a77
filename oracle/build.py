"""Build the plain-C FP64 oracle (oracle/liboracle.so).

Test infrastructure only: the library this builds is the checker that the
CUDA path is compared against; the product path never loads it.
Flags: -O2 without fast-math and with FMA contraction off, so that the FP32
cloud-in-cell index arithmetic is rounded exactly as written.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mg_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-fPIC", "-shared", SRC, "-o", LIB + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
