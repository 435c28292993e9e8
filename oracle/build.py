"""Compile the C oracle (oracle/ft_oracle.c) into oracle/libftoracle.so with gcc + OpenMP.

-ffp-contract=off keeps every multiply-add exactly as written: the oracle's pinned FP64
operation order only uses fma() where the source calls it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ft_oracle.c")
SRCS = [SRC, os.path.join(HERE, "ft_oracle_inj.c"), os.path.join(HERE, "ft_oracle_bin.c")]
LIB = os.path.join(HERE, "libftoracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and all(
            os.path.getmtime(LIB) >= os.path.getmtime(s) for s in SRCS):
        return LIB
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-std=gnu11"] + SRCS + ["-o", LIB + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
