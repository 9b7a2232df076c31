"""Compile the FP64 CPU oracle (test infrastructure) into oracle/liboracle.so.

Plain C, double precision, no fused multiply-add contraction, OpenMP over
cells where the compiler supports it.  Building the checker is not using it:
``__graft_entry__.build()`` calls this so that the oracle exists wherever the
tests run.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

BASE_FLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Build liboracle.so if it is missing or older than its source; return its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc"] + BASE_FLAGS + ["-fopenmp", SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(cmd, check=True, capture_output=True, text=True)
    except subprocess.CalledProcessError:
        # OpenMP is optional: the per-cell update has no reductions, so the
        # result does not depend on the thread count.
        cmd = ["gcc"] + BASE_FLAGS + [SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
