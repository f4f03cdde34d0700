"""Compile the FP64 C oracle into oracle/_bfgc_oracle.so.

Test infrastructure only (see oracle/__init__.py).  Plain gcc, no CUDA; OpenMP
is used when the compiler supports it, otherwise the oracle runs on one thread.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bfgc_oracle.c")
LIB = os.path.join(HERE, "_bfgc_oracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    """Build the oracle shared library if it is missing or older than its source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = os.environ.get("CC", "gcc")
    base = [cc, "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math", SRC, "-o", LIB + ".tmp", "-lm"]
    for extra in (["-fopenmp"], []):
        cmd = base[:1] + extra + base[1:]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(LIB + ".tmp", LIB)
            if verbose:
                print(" ".join(cmd))
            return LIB
        if verbose:
            print(r.stderr, file=sys.stderr)
    raise RuntimeError("could not compile the oracle: " + r.stderr)


if __name__ == "__main__":
    print(build(force=True, verbose=True))
