"""Compile the plain-C oracle (cholref.c) into liboracle_cholref.so with gcc.

Test infrastructure only: the CUDA library never links or loads the result.
Flags follow the oracle's contract: -O2, no fused multiply-add contraction,
no fast-math; OpenMP only splits independent rows across threads.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cholref.c")
LIB = os.path.join(HERE, "liboracle_cholref.so")


def build(force: bool = False, quiet: bool = True) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-std=c11", SRC, "-o", LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=quiet)
    except subprocess.CalledProcessError:
        # OpenMP is optional: the oracle is single-threaded without it.
        subprocess.run(base, check=True, capture_output=quiet)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, quiet=False))
