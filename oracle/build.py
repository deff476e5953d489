"""Build the FP64 oracle shared library (test infrastructure) with gcc + OpenMP."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def compile_library(src: str, out: str) -> str:
    """Compile a C source of the oracle into a shared library with the oracle's flags."""
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
           "-D_GNU_SOURCE", "-Wall", src, "-o", out, "-lm"]
    subprocess.check_call(cmd)
    return out


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    return compile_library(SRC, LIB)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
