"""Compile the oracle (plain C) into oracle/liboracle.so with the host gcc.

Building the checker is part of ``__graft_entry__.build()``; running it is
reserved to the tests, smoke() and bench.py's CPU baseline.
"""
from __future__ import annotations

import os
import platform
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "sv_oracle.c")
LIB = os.path.join(_HERE, "liboracle.so")


STAMP = os.path.join(_HERE, ".liboracle.arch")


def build(force: bool = False) -> str:
    here = platform.machine()
    same_arch = os.path.exists(STAMP) and open(STAMP).read().strip() == here
    if (not force and same_arch and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-fopenmp", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        f.write(here)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
