"""The device code's topology test, run on the host (no GPU).  The stage kernel decides
E_topo of Eq. equa:energy1 with a closed form (simple_mask: the label's ring cells that
are 4-neighbours of the block lie in one cyclic run of the 3x3 ring).  The function is
compiled here as host code from the library's own header and evaluated on all 256 masks.
It must equal the oracle's breadth-first search, and the classical (4,8) simple-point
definition everywhere except the full ring."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from test_oracle_bruteforce import simple_classical

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1704_02083_gb300", "csrc")
RING = [(-1, -1), (0, -1), (1, -1), (1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0)]


@pytest.fixture(scope="module")
def device_table(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("host_topology")
    src = d / "table.cu"
    src.write_text('#include <stdio.h>\n#include "rapid_dev.cuh"\n'
                   "int main(void) { for (unsigned m = 0; m < 256; m++) printf(\"%d\", rapid::simple_mask(m) ? 1 : 0);"
                   ' printf("\\n"); return 0; }\n')
    exe = d / "table"
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                    "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True, timeout=600)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True, timeout=60).stdout.strip()
    assert len(out) == 256
    return np.array([int(c) for c in out], np.uint8)


def test_device_topology_equals_the_oracle(device_table):
    np.testing.assert_array_equal(device_table, oracle.simple_lut())


def test_device_topology_against_the_classical_definition(device_table):
    for m in range(256):
        g = np.zeros((3, 3), np.int32)
        g[1, 1] = 1
        for i, (dx, dy) in enumerate(RING):
            if m >> i & 1:
                g[1 + dy, 1 + dx] = 1
        want = simple_classical(g, 1, 1) if m != 0xFF else True
        assert bool(device_table[m]) == bool(want), hex(m)
