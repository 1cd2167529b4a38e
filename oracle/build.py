"""Compile the oracle's C exact solver (``oracle/ssp.c``) into a shared library.

TEST INFRASTRUCTURE ONLY: building the checker is not using it.  The library
lands in ``oracle/_build/`` (git-ignored) so that each machine builds its own.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ssp.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle_ssp.so")


def build(force: bool = False) -> str:
    """Build ``liboracle_ssp.so`` if it is missing or older than its source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC",
                           SRC, "-o", tmp, "-lm"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
