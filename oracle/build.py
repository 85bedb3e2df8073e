"""Compile the oracle's plain-C direct sums (TEST INFRASTRUCTURE ONLY).

``python -m oracle.build`` (or ``build()``) writes ``oracle/_direct_sum.so`` with
gcc -O2 -fopenmp.  Building the checker is not using it: the product library
never links or loads this file.
"""

from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "direct_sum.c")
LIB = os.path.join(HERE, "_direct_sum.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
