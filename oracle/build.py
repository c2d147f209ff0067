"""Build the CPU oracle (test infrastructure) as oracle/_build/liboracle.so.

Flags: -O2 with -ffp-contract=off and no fast-math, so every double operation of the
oracle is a separately rounded IEEE operation in source order on x86-64 and AArch64 alike.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
LIB_OMP = os.path.join(OUT_DIR, "liboracle_omp.so")  # the same source, phase decisions on all cores
SRC = [os.path.join(HERE, "rapid_oracle.c")]
HDR = [os.path.join(HERE, "rapid_oracle.h")]


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in SRC + HDR + [__file__])


def compile_to(out: str, sources=SRC, openmp: bool = False) -> str:
    """Compile the oracle's C sources into the shared library ``out`` (with ``openmp`` the
    decisions of a phase run on all cores: -fopenmp -DORC_OPENMP)."""
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-Wno-unused-parameter"] + (["-fopenmp", "-DORC_OPENMP"] if openmp else []) + \
          ["-o", out] + list(sources) + ["-lm"]
    subprocess.run(cmd, check=True)
    return out


def build(force: bool = False, openmp: bool = False) -> str:
    lib = LIB_OMP if openmp else LIB
    if not force and not _stale(lib):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = lib + f".tmp{os.getpid()}"
    compile_to(tmp, openmp=openmp)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True), build(force=True, openmp=True))
