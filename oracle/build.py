"""Compile the CPU oracle (test infrastructure) into oracle/_build/liboracle.so.

Only the test suite, the package smoke check and the benchmark's CPU-baseline
leg load the result. Host-portable flags only: the same source builds on x86_64
and aarch64.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "im_oracle.cpp")
OUT_DIR = os.path.join(HERE, "_build")
OUT = os.path.join(OUT_DIR, "liboracle.so")
OUT_OMP = os.path.join(OUT_DIR, "liboracle_omp.so")


def _compile(out, extra, force):
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC"] + extra + ["-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Single-threaded oracle (the default for every test)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    return _compile(OUT, [], force)


def build_omp(force: bool = False) -> str:
    """The same source with OpenMP: all host cores, identical results."""
    os.makedirs(OUT_DIR, exist_ok=True)
    return _compile(OUT_OMP, ["-fopenmp"], force)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build_omp(force="--force" in sys.argv))
