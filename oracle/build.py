"""Compile the FP64 CPU oracle (test infrastructure) into a shared library.

Plain gcc, -O2 with floating-point contraction off so that every multiply and add is
rounded separately, exactly as the C source reads.  OpenMP (-fopenmp) shares the independent
row and point loops among threads when the compiler supports it; the results do not depend on
the thread count, and without OpenMP the same source builds as a single-threaded library.
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
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-Wall", "-Wextra", "-o", tmp, SOURCE, "-lm"]
    for cmd in (base[:1] + ["-fopenmp"] + base[1:], base):
        if verbose:
            print(" ".join(cmd))
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            break
        if verbose:
            print(f"(failed: {r.stderr.strip()[:300]})")
    else:
        raise RuntimeError(f"gcc failed on {SOURCE}:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
