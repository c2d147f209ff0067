"""The C ABI library: it builds for sm_103a, loads without a GPU, and exports every
function include/rapid.h declares; struct layouts agree between the header and the
binding.  No CUDA compute call is made here."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rapid.h")


@pytest.fixture(scope="module")
def pkg():
    from paper_1704_02083_gb300 import build
    build.build()
    import paper_1704_02083_gb300 as p
    p.lib()
    return p


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(rapid_[a-z_]+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("rapid_create", "rapid_set_image", "rapid_seed_grid", "rapid_refine_stage", "rapid_split",
              "rapid_run", "rapid_read_labels", "rapid_read_stats", "rapid_read_counters", "rapid_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(pkg):
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(rapid_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = pkg.lib()
    for n in declared_functions():
        assert hasattr(lib, n)


def test_binding_has_the_c_names(pkg):
    for n in declared_functions():
        assert callable(getattr(pkg, n)), n


def test_host_only_calls(pkg):
    assert pkg.rapid_status_string(0) == "RAPID_OK"
    assert "device wait" in pkg.rapid_status_string(5)
    assert pkg.rapid_status_string(99).startswith("RAPID_?")
    p = pkg.rapid_default_params()
    assert (p.num_levels, p.ratio_C, p.init_block, p.final_grain, p.K, p.size_mode) == (1, 4, 16, 1, 200, 2)
    assert (p.lambda_pos0, p.lambda_b) == (400.0, 50.0)
    assert (p.lo_num, p.lo_den, p.hi_num, p.hi_den) == (1, 4, 3, 2)
    assert (p.max_sweeps, p.h_T, p.spin_limit_ns) == (64, 150, 2_000_000_000)
    assert (p.use_filter, p.skip_tiles, p.verify_filter) == (1, 1, 0)
    with pytest.raises(pkg.RapidError) as e:  # argument check happens before any CUDA call
        pkg.rapid_create(pkg.rapid_default_params(K=0))
    assert e.value.status == pkg.RAPID_EINVAL


def test_struct_layouts_match_header(pkg, tmp_path):
    probe = tmp_path / "probe.c"
    probe.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "rapid.h"\nint main(void){'
                     'printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(rapid_params), sizeof(rapid_sp_stats),'
                     ' sizeof(rapid_stage_counters), sizeof(rapid_counters), offsetof(rapid_params, h_T),'
                     ' offsetof(rapid_counters, stage));return 0;}\n')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()))
    want = [C.sizeof(pkg.rapid_params), C.sizeof(pkg.rapid_sp_stats), C.sizeof(pkg.rapid_stage_counters),
            C.sizeof(pkg.rapid_counters), pkg.rapid_params.h_T.offset, pkg.rapid_counters.stage.offset]
    assert got == want
