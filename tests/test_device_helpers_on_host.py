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


def _host_program(tmp_path_factory, name, body):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp(name)
    src = d / "prog.cu"
    src.write_text('#include <stdio.h>\n#include "rapid_dev.cuh"\nint main(void) {\n' + body + "\nreturn 0; }\n")
    exe = d / "prog"
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                    "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True, timeout=600)
    return subprocess.run([str(exe)], capture_output=True, text=True, check=True, timeout=60).stdout.split()


def test_select_bit_finds_every_set_bit(tmp_path_factory):
    """select_bit(m, k), which spreads a word's set bits over the lanes of the sweep walk,
    gives the position of the k-th set bit for every k of 2000 pseudo-random words and
    the edge words (one bit, all bits)."""
    words = [1, 0x80000000, 0xFFFFFFFF, 0x55555555, 0xAAAAAAAA]
    x = 12345
    for _ in range(2000):
        x = (x * 6364136223846793005 + 1442695040888963407) % (1 << 64)
        words.append((x >> 32) | 1)
    body = "const unsigned w[] = {" + ",".join(f"{v}u" for v in words) + "};\n" \
           f"for (int i = 0; i < {len(words)}; i++) for (int k = 0; k < rapid::popc32(w[i]); k++)" \
           ' printf("%d ", rapid::select_bit(w[i], k));'
    got = [int(v) for v in _host_program(tmp_path_factory, "select_bit", body)]
    want = [p for v in words for p in range(32) if v >> p & 1]
    assert got == want


def test_class_lattice_covers_every_block_once(tmp_path_factory):
    """The sweep schedule's bitmap geometry: over the 9 phase classes, the lattice columns
    (class_cols) and rows (class_rows) of a grid hold every block exactly once, and a row of
    class_wpr words has room for its columns, for grids from 1 x 1 up to odd large sides."""
    sizes = [(1, 1), (1, 7), (7, 1), (2, 2), (3, 3), (4, 5), (95, 96), (97, 33), (1366, 1), (4096, 4096)]
    body = "const int s[][2] = {" + ",".join(f"{{{a},{b}}}" for a, b in sizes) + "};\n" \
           f"for (int i = 0; i < {len(sizes)}; i++) for (int c = 0; c < 9; c++)" \
           ' printf("%d %d %d %lld ", rapid::class_cols(s[i][0], c % 3), rapid::class_rows(s[i][1], c / 3),' \
           " rapid::class_wpr(s[i][0], c % 3), rapid::class_words(s[i][0], s[i][1], c));"
    out = [int(v) for v in _host_program(tmp_path_factory, "class_lattice", body)]
    it = iter(out)
    for nbx, nby in sizes:
        total = 0
        for c in range(9):
            cols, rows, wpr, words = next(it), next(it), next(it), next(it)
            px, py = c % 3, c // 3
            assert cols == len(range(px, nbx, 3)) and rows == len(range(py, nby, 3))
            assert wpr * 32 >= cols > (wpr - 1) * 32 or (cols == 0 and wpr == 0)
            assert words == rows * wpr
            total += cols * rows
        assert total == nbx * nby
