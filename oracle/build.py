"""Compile the plain-C oracle (test infrastructure) into a shared library.

gcc -O2 -fPIC -shared -ffp-contract=off [-fopenmp]: no fast-math and no FMA
contraction, so the oracle rounds every product and sum separately on every
host architecture.  OpenMP (when available) only parallelises independent
rows of the CSR/ELL SpMV loops.
"""
from __future__ import annotations

import os
import subprocess
import sys

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "gko_oracle.c")


def lib_path() -> str:
    return os.path.join(_HERE, "liboracle.so")


def build(verbose: bool = False) -> str:
    out = lib_path()
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
            "-fno-fast-math", SRC, "-o", out + ".tmp", "-lm"]
    for extra in (["-fopenmp"], []):
        cmd = base[:4] + extra + base[4:]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(out + ".tmp", out)
            if verbose:
                print(" ".join(cmd))
            return out
    sys.stderr.write(r.stderr)
    raise RuntimeError("oracle build failed")


if __name__ == "__main__":
    print(build(verbose=True))
