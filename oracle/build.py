"""Compile the C++ oracle into oracle/libxfo.so (test infrastructure only)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "xfo.cpp")
LIB = os.path.join(HERE, "libxfo.so")
# -ffp-contract=off keeps every multiply and add separately rounded, as written
FLAGS = ["-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC),
                                             os.path.getmtime(os.path.join(HERE, "xfo.h")))):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", *FLAGS, "-o", tmp, SRC])
    os.replace(tmp, LIB)
    return LIB


def compile_source(src: str, out: str) -> str:
    """Compile an oracle source file ``src`` (e.g. a copy with a planted
    mistake, made by a test) into the shared library ``out`` with the same
    flags as the oracle itself."""
    subprocess.check_call(["g++", *FLAGS, "-I", HERE, "-o", out, src])
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
