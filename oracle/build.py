"""Compile the C oracle into ``oracle/_build/liboracle.so`` with gcc (OpenMP when available).

Part of the test infrastructure: the product library never builds or loads this.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def _compile(flags):
    os.makedirs(OUT_DIR, exist_ok=True)
    fd, tmp = tempfile.mkstemp(prefix="liboracle.", suffix=".so", dir=OUT_DIR)
    os.close(fd)
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", *flags, SRC, "-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        os.unlink(tmp)
        return r.stderr
    os.replace(tmp, LIB)  # atomic: concurrent builders never see a half-written library
    return None


def build(force: bool = False) -> str:
    """Build the oracle if missing or stale; returns the library path."""
    if (not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    if shutil.which("gcc") is None:
        raise RuntimeError("gcc not found: cannot build the oracle")
    err = _compile(["-fopenmp"])
    if err is not None:
        err2 = _compile([])
        if err2 is not None:
            raise RuntimeError("oracle build failed:\n" + err + "\n" + err2)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
