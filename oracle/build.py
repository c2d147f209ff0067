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
SRC = [os.path.join(HERE, "rapid_oracle.c")]
HDR = [os.path.join(HERE, "rapid_oracle.h")]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in SRC + HDR + [__file__])


def compile_to(out: str, sources=SRC) -> str:
    """Compile the oracle's C sources into the shared library ``out``."""
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-Wno-unused-parameter", "-o", out] + list(sources) + ["-lm"]
    subprocess.run(cmd, check=True)
    return out


def build(force: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    compile_to(tmp)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
