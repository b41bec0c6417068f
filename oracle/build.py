"""Compile the C oracle into ``oracle/_tc_oracle.so`` with gcc.

TEST INFRASTRUCTURE: this builds the checker, nothing in the product path
loads it.  Plain gcc, no architecture flags, so the same source builds on the
x86_64 development host and on an aarch64 host.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tc_oracle.c")
LIB = os.path.join(HERE, "_tc_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
