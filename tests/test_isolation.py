"""Separation of the library from its checker, checked on the sources (no GPU):
  * nothing in the package (Python, CUDA, headers) imports, includes or loads the oracle;
  * the oracle includes no header of the library and no file of the package;
  * the only module both sides import is the seeded input generator, which imports neither;
  * without the built library the package fails loudly instead of falling back to a CPU
    path."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1704_02083_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _sources(top, exts):
    for d, _, files in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def _code(path):
    """Source text without comments and docstrings (a citation may name the oracle)."""
    src = open(path).read()
    if path.endswith(".py"):
        src = re.sub(r'("""|\'\'\').*?\1', "", src, flags=re.S)
        return "\n".join(line.split("#", 1)[0] for line in src.splitlines())
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return "\n".join(line.split("//", 1)[0] for line in src.splitlines())


def test_package_never_reaches_the_oracle():
    bad = re.compile(r"\boracle\b|rapid_oracle|liboracle|orc_[a-z]")
    hits = [(p, m.group(0)) for p in _sources(PKG, (".py", ".cu", ".cuh", ".h", ".cpp"))
            for m in [bad.search(_code(p))] if m]
    assert not hits, hits


def test_oracle_includes_nothing_of_the_library():
    for p in _sources(ORACLE, (".c", ".h")):
        src = open(p).read()
        local = re.findall(r'#\s*include\s*"([^"]+)"', src)  # quoted: this project's own headers
        assert local in ([], ["rapid_oracle.h"]), (p, local)
        system = re.findall(r'#\s*include\s*<([^>]+)>', src)  # C library and OpenMP only
        assert all(i.split(".")[0] in ("stdint", "stdio", "stdlib", "string", "math", "omp", "stddef", "limits")
                   for i in system), (p, system)
    for p in _sources(ORACLE, (".py",)):
        code = _code(p)
        assert "paper_1704_02083_gb300" not in code and "librapid" not in code, p


def test_shared_input_generator_imports_neither_side():
    code = _code(os.path.join(PKG, "synth.py"))
    imports = re.findall(r"^\s*(?:from\s+(\S+)\s+import|import\s+(\S+))", code, re.M)
    names = {a or b for a, b in imports}
    assert names and all(n.split(".")[0] in {"__future__", "dataclasses", "numpy", "scipy", "os", "math", "typing"}
                         for n in names), names


def test_missing_library_fails_loudly(tmp_path):
    """A fresh interpreter whose package points at a library that is not there: the first
    call raises ImportError; nothing computes on the CPU instead."""
    prog = (
        "import sys; sys.path.insert(0, %r)\n"
        "import paper_1704_02083_gb300 as p\n"
        "p.LIB_PATH = %r\n"
        "p._lib = None\n"
        "try:\n"
        "    p.rapid_status_string(0)\n"
        "except ImportError as e:\n"
        "    print('raised', 'no CPU fallback' in str(e))\n"
        "else:\n"
        "    print('no error')\n" % (ROOT, str(tmp_path / "librapid.so")))
    out = subprocess.run([sys.executable, "-c", prog], capture_output=True, text=True, timeout=300)
    assert out.stdout.strip() == "raised True", out.stdout + out.stderr


def test_stored_expected_values_come_from_the_oracle_alone():
    """The script that writes tests/golden/ imports the oracle and the input generator and
    nothing of the CUDA path."""
    code = _code(os.path.join(ROOT, "tests", "golden", "make_golden.py"))
    imports = re.findall(r"^\s*(?:from\s+(\S+)\s+import\s+(.+)|import\s+(\S+))", code, re.M)
    mods = {(a, b.strip()) if a else (c, "") for a, b, c in imports}
    pkg_imports = {m for m in mods if m[0].startswith("paper_1704_02083_gb300")}
    assert pkg_imports == {("paper_1704_02083_gb300", "synth")}, pkg_imports
    assert ("oracle", "") in mods
    assert "librapid" not in code and "Context(" not in code and "rapid_" not in code
