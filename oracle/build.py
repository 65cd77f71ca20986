"""Build the CPU oracle shared library (test infrastructure only).

Compiles ``twopaco_oracle.cpp`` with the host C++ compiler into
``liboracle.so`` beside it. Portable C++17: no target-specific flags, so it
builds the same way on x86_64 and aarch64 hosts.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "twopaco_oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")


MUTANT_DIR = os.path.join(os.path.dirname(HERE), "_build", "oracle_mutants")


def build_mutant(n: int, force: bool = False) -> str:
    """A test build of the oracle with planted mistake n (ORACLE_MUTANT = n), for checking
    that the pins catch it; never loaded outside the tests."""
    os.makedirs(MUTANT_DIR, exist_ok=True)
    lib = os.path.join(MUTANT_DIR, f"liboracle_mutant{n}.so")
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    cmd = [os.environ.get("CXX", "g++"), "-std=c++17", "-O1", "-shared", "-fPIC", "-pthread",
           f"-DORACLE_MUTANT={int(n)}", "-o", lib + ".tmp", SRC]
    subprocess.run(cmd, check=True)
    os.replace(lib + ".tmp", lib)
    return lib


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = [os.environ.get("CXX", "g++"), "-std=c++17", "-O2", "-shared", "-fPIC", "-pthread",
           "-o", LIB + ".tmp", SRC]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
