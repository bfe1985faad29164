"""Build the FP64 CPU oracle (test infrastructure) with gcc.

Plain C, -O2, no fast-math and no floating-point contraction, so the oracle
evaluates each formula as written. The shared library lands beside the source
(git-ignored) and is rebuilt when the source is newer.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "relsim_oracle.c")
SRC3 = os.path.join(HERE, "relsim_oracle3.c")
SRCQ = os.path.join(HERE, "relsim_oracle_q.c")


def lib_path() -> str:
    return os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    out = lib_path()
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(SRC)
            and os.path.getmtime(out) >= os.path.getmtime(SRC3)
            and os.path.getmtime(out) >= os.path.getmtime(SRCQ)
            and os.path.getmtime(out) >= os.path.getmtime(os.path.join(HERE, "relsim_oracle.h"))):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, SRC, SRC3, SRCQ, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
