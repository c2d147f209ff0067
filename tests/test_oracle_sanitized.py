"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer.

A copy built with -fsanitize=address,undefined refines the edge cases: 1 x 1, a single
row, a single column, more superpixels than blocks, a grain above the initial block,
three levels with either importance rule, both schedules, the FIFO variant and the
classifier.  It also refines the 321 x 481 workload.  Every run goes through a separate
interpreter with the sanitizer runtimes preloaded, and any report ends it with an error.
The checker must not read or write out of bounds or rely on undefined behaviour: its
results are the reference for everything else."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ORACLE_DIR = os.path.join(ROOT, "oracle")

CASES = [(1, 1, dict(K=1)), (1, 37, dict(K=3, init_block=8)), (37, 1, dict(K=3, init_block=8)),
         (5, 7, dict(K=40, init_block=4)), (33, 47, dict(K=9, init_block=4, num_levels=2, ratio_C=4, predict=1)),
         (64, 48, dict(K=16, init_block=16, num_levels=3, ratio_C=2, predict=1, importance_rule=1)),
         (96, 80, dict(K=24, init_block=16, num_levels=3, ratio_C=4, predict=1, schedule=1)),
         (50, 70, dict(K=30, init_block=8, final_grain=2, size_mode=1)),
         (8, 8, dict(K=4, init_block=32, final_grain=64))]


def _runtime(name):
    p = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
    return p if os.path.isabs(p) and os.path.exists(p) else None


def test_oracle_is_clean_under_sanitizers(tmp_path):
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not (asan and ubsan):
        pytest.skip("gcc's sanitizer runtimes are not installed")
    lib = str(tmp_path / "liboracle_san.so")
    subprocess.run(["gcc", "-std=c11", "-O1", "-g", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer",
                    "-o", lib, os.path.join(ORACLE_DIR, "rapid_oracle.c"), "-lm"], check=True, timeout=300)
    env = dict(os.environ, LD_PRELOAD=f"{asan} {ubsan}", ASAN_OPTIONS="detect_leaks=0:halt_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), lib], env=env, capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0 and "sanitized runs: ok" in r.stdout, (r.stdout + r.stderr)[-4000:]


def _child(lib):
    for p in (ROOT, ORACLE_DIR, HERE):
        sys.path.insert(0, p)
    import oracle
    from paper_1704_02083_gb300 import synth

    oracle._build.build = lambda force=False: lib
    assert oracle.lib()._name == lib
    for H, W, p in CASES:
        for seed in range(3):
            rgb = synth.he_image(H, W, 3, seed).rgb
            o = oracle.Oracle(rgb, **p).run()
            o.labels(), o.stats(), o.counters()
            oracle.Oracle(rgb, **p).run_fifo().labels()
            oracle.Oracle(rgb, **p).set_classifier([1.0, -0.01, 0.1, 0.2, 0.3]).run().features()
    w = synth.WORKLOADS["he321x481_k200"]
    oracle.Oracle(synth.workload_image("he321x481_k200").rgb, **w["params"]).run().labels()
    print("sanitized runs: ok")


if __name__ == "__main__":
    _child(sys.argv[1])
