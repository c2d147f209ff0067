"""Build the CUDA library in-tree: paper_1704_02083_gb300/_build/librapid.so (sm_103a).

Every translation unit is compiled for sm_103a only, with -fmad=false (no contraction of
double multiply-adds anywhere) and -ffp-contract=off for host code, then linked into one
shared library with the static CUDA runtime.  Translation units compile in parallel.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "librapid.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
UNITS = ["k_stage_s0.cu", "k_stage_s1.cu", "k_stage_s2.cu", "k_stage_s3.cu", "k_stage_s4.cu", "k_stage_s5.cu",
         "k_stage.cu", "k_prep.cu", "k_scorer.cu",
         "rapid_api.cu", "rapid_static.cu", "k_synth.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-fmad=false", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "-I" + INCLUDE]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return p


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return files + [__file__]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    tag = f"{os.getpid()}"

    def compile_one(u):
        obj = os.path.join(OUT_DIR, u.replace(".cu", f".{tag}.o"))
        cmd = [cc] + NVCC_FLAGS + ["-c", os.path.join(CSRC, u), "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {u}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + f".tmp{tag}"
    r = subprocess.run([cc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs, capture_output=True,
                       text=True)
    for o in objs:
        try:
            os.remove(o)
        except OSError:
            pass
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
