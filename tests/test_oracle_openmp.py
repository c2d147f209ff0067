"""The oracle's all-core build (the decisions of a phase on OpenMP threads, the CPU
baseline on every host core): the same labels, statistics, classes, importance flags and
counters as the single-threaded oracle, for any thread count.  The blocks of a phase decide
independently (disjoint windows, the phase snapshot) and their outcomes are listed in block
order, so no result may depend on the threads."""
import os

import numpy as np
import pytest

import oracle
from paper_1704_02083_gb300 import synth

CASES = [
    ("bsd321x481", lambda: synth.workload_image("he321x481_k200").rgb,
     dict(synth.WORKLOADS["he321x481_k200"]["params"])),
    ("he256_l3", lambda: synth.he_image(256, 256, 30, 21).rgb,
     dict(num_levels=3, ratio_C=4, init_block=32, K=64, size_mode=2, predict=1)),
    ("rand61x47_rule1", lambda: synth.random_image(61, 47, 8, levels=5),
     dict(num_levels=2, ratio_C=2, init_block=8, K=20, size_mode=1, predict=1, importance_rule=1, reuse=0)),
    ("he200_queue", lambda: synth.he_image(200, 150, 12, 22).rgb,
     dict(num_levels=2, ratio_C=4, init_block=16, K=40, size_mode=2, predict=1, schedule=1)),
]


def _all(o):
    s, y, imp = o.stats()
    return o.labels(), s, y, imp, o.counters()


@pytest.mark.parametrize("name,img,params", CASES, ids=[c[0] for c in CASES])
def test_all_core_oracle_equals_the_single_thread_oracle(name, img, params):
    rgb = img()
    want = _all(oracle.Oracle(rgb, **params).run())
    for threads in sorted({1, 2, 3, 8, os.cpu_count() or 1}):
        got = _all(oracle.Oracle(rgb, omp=True, threads=threads, **params).run())
        for a, b, what in zip(got, want, ("labels", "S", "y", "importance", "counters")):
            np.testing.assert_array_equal(a, b, err_msg=f"{name}, {threads} threads: {what}")


def test_all_core_oracle_uses_the_threads_it_is_given():
    o = oracle.Oracle(np.zeros((8, 8, 3), np.uint8), omp=True, threads=3)
    assert o.threads == 3
