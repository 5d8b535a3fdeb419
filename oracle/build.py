"""Compile the C oracle into ``oracle/_build/liboracle.so`` (test infrastructure).

``-ffp-contract=off`` is required: the oracle evaluates the k-means distances
in binary32 in a fixed order without fused multiply-adds.  ``-fopenmp`` is for
``gira_oracle_par.c`` (the EM iteration over all host cores); the
single-threaded functions of ``gira_oracle.c`` hold no OpenMP directive.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "gira_oracle.c"), os.path.join(HERE, "gira_oracle_par.c")]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")

CFLAGS = ["-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
          "-Wall", "-Wextra", "-Werror", "-fopenmp"]


def build(force: bool = False) -> str:
    """Build the shared library if missing or older than its source; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in SRCS):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, "-o", tmp, *SRCS, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
