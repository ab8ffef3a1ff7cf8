"""Compile the FP64 CPU oracle (plain C, gcc + OpenMP) into oracle/_build/.

Test infrastructure only: the shared library this builds is loaded by the
tests, the smoke check and the CPU baseline, never by the solver.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pfm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Build liboracle.so if missing or older than its source; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    newest_src = max(os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "pfm_oracle.h")))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest_src:
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
