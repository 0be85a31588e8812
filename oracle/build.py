"""Compile the CPU oracle (test infrastructure).

oracle/liboracle.so is the serial parity reference; oracle/liboracle_omp.so
is the same source compiled with -fopenmp, the all-cores timing baseline.
Plain gcc, FP64, no FMA contraction, no architecture flags, so the same
source gives the same results on x86-64 and aarch64 hosts.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "airga_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
LIB_OMP = os.path.join(HERE, "liboracle_omp.so")


def _compile(out: str, extra: list[str], force: bool) -> str:
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           *extra, "-shared", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False, openmp: bool = False) -> str:
    """Path of the serial library (openmp=False) or of the OpenMP one."""
    if openmp:
        return _compile(LIB_OMP, ["-fopenmp"], force)
    return _compile(LIB, [], force)


def build_all(force: bool = False) -> list[str]:
    return [build(force), build(force, openmp=True)]


if __name__ == "__main__":
    print(build_all(force="--force" in sys.argv))
