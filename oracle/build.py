"""Compile the C oracle (oracle.c) into oracle/liboracle.so.

TEST INFRASTRUCTURE ONLY: the library built here is loaded by the tests, the
smoke check and the benchmark's CPU-baseline leg, never by the product path.
Plain gcc, no architecture-specific flags, so the same source builds on the
x86 development host and the aarch64 GPU host.
"""

from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False, plant: int = 0, out: str | None = None) -> str:
    """Build the oracle library.  ``plant`` > 0 builds a variant with one
    deliberate mistake (see ORACLE_PLANT in oracle.c) into ``out``; only the
    tests that show the pins catching mistakes ask for one."""
    lib = out or LIB
    if plant == 0 and not force and os.path.exists(lib) \
            and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=gnu11",
           f"-DORACLE_PLANT={int(plant)}", "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
