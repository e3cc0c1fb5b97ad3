"""Build the CPU oracle (TEST INFRASTRUCTURE ONLY) into oracle/liboracle.so.

Plain gcc, no fast-math and no floating-point contraction, so every + - * of
Eq. 3 is one IEEE round-to-nearest operation on both x86_64 and aarch64 (gcc
contracts a*b+c into an FMA by default on aarch64; -ffp-contract=off stops it).
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["tcm_oracle.c", "tcm_oracle_impl.inc", "tcm_oracle.h"]
LIB = os.path.join(HERE, "liboracle.so")
BASE_FLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
              "-Wall", "-Wextra"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in SOURCES)


def build(force: bool = False) -> str:
    """Compile the oracle if its sources are newer than the library."""
    if not force and not _stale():
        return LIB
    src = os.path.join(HERE, "tcm_oracle.c")
    tmp = LIB + f".tmp{os.getpid()}"
    for extra in (["-fopenmp"], []):
        cmd = ["gcc", *BASE_FLAGS, *extra, "-o", tmp, src, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, LIB)
            return LIB
    raise RuntimeError("oracle build failed:\n" + r.stderr)


if __name__ == "__main__":
    print(build(force=True))
