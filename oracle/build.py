"""Compile the CPU oracle (plain C, FP64) into oracle/liboracle.so.

Test infrastructure: only the test-suite, the smoke check and the CPU baseline leg of
the benchmark load the result.  FP contraction is off so that x86 and Arm hosts round
identically.  OpenMP runs the loops over independent groups (or cells) on several threads
for the CPU baseline; the results do not depend on the thread count.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["physics.c", "sweep.c", "lo.c", "driver.c"]
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES] + [os.path.join(HERE, "oracle.h")]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-Wall", "-fopenmp",
           "-shared", "-fPIC", "-o", LIB + ".tmp"]
    cmd += [os.path.join(HERE, s) for s in SOURCES] + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
