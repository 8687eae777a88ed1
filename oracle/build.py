"""Compile the FP64 CPU oracle (``lbm_oracle.c``) into ``oracle/_lib/liblbm_oracle.so``.

Test infrastructure only: the oracle checks the CUDA library, it is never part of it.
Plain gcc, ``-O2 -ffp-contract=off`` so x86 and Arm hosts round identically, OpenMP over
z-planes when the compiler supports it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
OUT_DIR = os.path.join(HERE, "_lib")
OUT = os.path.join(OUT_DIR, "liblbm_oracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    """Build the oracle shared library if it is missing or older than its source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= os.path.getmtime(SRC):
        return OUT
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", SRC, "-lm"]
    tmp = OUT + f".tmp{os.getpid()}"
    cmd = base[:-1] + ["-fopenmp", "-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:  # no OpenMP: build single-threaded
        cmd = base + ["-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"oracle build failed: {' '.join(cmd)}\n{r.stderr}")
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True, verbose=True))
