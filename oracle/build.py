"""Compile the C oracle (oracle.c) into oracle/liboracle.so with gcc (with
OpenMP when available, for or_set_threads).

Test infrastructure only.  -ffp-contract=off keeps the written arithmetic
(no fused multiply-add contraction), so the oracle computes what it states.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SOURCES = [os.path.join(HERE, "oracle.c"), os.path.join(HERE, "unet_oracle.c")]


def build(force: bool = False) -> str:
    srcs = [s for s in SOURCES if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(HERE, "oracle.h")])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-o", tmp] + srcs + ["-lm"]
    # OpenMP (or_set_threads) where the compiler has it; a build without it
    # runs every loop on one thread and computes the same bits.
    try:
        subprocess.check_call(cmd[:1] + ["-fopenmp"] + cmd[1:], stderr=subprocess.DEVNULL)
    except (subprocess.CalledProcessError, OSError):
        subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
