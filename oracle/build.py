"""Compile the FP64 CPU oracle (test infrastructure) into a shared library.

Plain gcc, -O2 with floating-point contraction off so that every multiply and add is
rounded separately, exactly as the C source reads.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(HERE, "raftgp_oracle.c")


def library_path() -> str:
    return os.path.join(HERE, "_build", "liboracle_raftgp.so")


def build(verbose: bool = False) -> str:
    out = library_path()
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-o", tmp, SOURCE, "-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
