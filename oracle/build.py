"""Builds the oracle's shared library (TEST INFRASTRUCTURE ONLY).

The oracle is plain C compiled with gcc, FMA contraction off so that x86 and Arm hosts round
identically.  It is built next to its source, under ``oracle/_build/``.  ``build(openmp=True)``
builds the same source with -fopenmp into ``liboracle_omp.so``, used only to time the oracle on
all host cores (its column loops run in parallel; every result is bitwise the serial one's).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tsqr_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
LIB_OMP = os.path.join(OUT_DIR, "liboracle_omp.so")


def build(force: bool = False, openmp: bool = False) -> str:
    """Compiles ``liboracle.so`` (or, with openmp, ``liboracle_omp.so``) if it is missing or older
    than its source; returns its path."""
    lib = LIB_OMP if openmp else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    cmd += ["-fopenmp"] if openmp else []
    cmd += ["-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True))
