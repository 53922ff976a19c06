"""Compile the oracle's C sources into shared libraries next to them.

Test infrastructure: the oracle (serial) and the all-core CPU baseline (OpenMP)
are only loaded by the test-suite, the smoke check and the CPU-baseline legs of
the benchmark.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "stencil_oracle.c")
LIB = os.path.join(HERE, "_liboracle.so")
OMP_SRC = os.path.join(HERE, "stencil_omp.c")
OMP_LIB = os.path.join(HERE, "_liboracle_omp.so")

# Every + and * must be one IEEE-754 operation: no contraction into FMA (the
# aarch64 compiler contracts by default), no fast-math reassociation.
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def _compile(src: str, lib: str, extra: list[str], force: bool) -> str:
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(src):
        return lib
    tmp = lib + ".tmp.%d" % os.getpid()
    subprocess.run(["gcc", *CFLAGS, *extra, "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    _compile(OMP_SRC, OMP_LIB, ["-fopenmp"], force)
    return _compile(SRC, LIB, [], force)


def build_omp(force: bool = False) -> str:
    return _compile(OMP_SRC, OMP_LIB, ["-fopenmp"], force)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
