"""GPU parity: label maps, statistics and per-stage counters of the CUDA path, called
through the C ABI, equal the CPU oracle's bit for bit (integer labels and int64 sums;
every decision is taken from binary64 energies in the same operation order on both
sides)."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from gpu_common import assert_parity, gpu_run, oracle_run
from paper_1704_02083_gb300 import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def test_topology_table_matches_oracle():
    import paper_1704_02083_gb300 as pkg
    np.testing.assert_array_equal(pkg.rapid_simple_table(), oracle.simple_lut())


def test_bsd_sized_image():
    """321 x 481, 200 requested superpixels, blocks 16 -> 1 (single level)."""
    w = synth.WORKLOADS["he321x481_k200"]
    img = synth.workload_image("he321x481_k200")
    lab, st, cnt = assert_parity(img.rgb, **w["params"])
    assert cnt[:, 5].sum() > 0 and cnt[:, 7].sum() > 0  # moves and merges happened


TINY = []
for seed in range(40):
    rng = np.random.default_rng(1000 + seed)
    H, W = int(rng.integers(1, 70)), int(rng.integers(1, 70))
    TINY.append(dict(H=H, W=W, seed=seed, K=int(rng.integers(1, 40)),
                     init_block=int(2 ** rng.integers(0, 5)), size_mode=int(rng.integers(0, 3)),
                     num_levels=int(rng.integers(1, 4)), ratio_C=int(2 ** rng.integers(1, 3)),
                     predict=int(rng.integers(0, 2)), reuse=int(rng.integers(0, 2)),
                     importance_rule=int(rng.integers(0, 2)), final_grain=int(2 ** rng.integers(0, 2)),
                     levels=int(rng.choice([2, 4, 256]))))


@pytest.mark.parametrize("case", TINY, ids=[f"t{i}" for i in range(len(TINY))])
def test_tiny_random(case):
    c = dict(case)
    H, W, seed, levels = c.pop("H"), c.pop("W"), c.pop("seed"), c.pop("levels")
    rgb = synth.random_image(H, W, seed, levels=levels) if seed % 2 else synth.he_image(H, W, 4, seed).rgb
    assert_parity(rgb, **c)


MID = [
    dict(H=200, W=264, cells=14, seed=21, num_levels=3, ratio_C=4, init_block=32, K=48, predict=1),
    dict(H=200, W=264, cells=14, seed=21, num_levels=3, ratio_C=4, init_block=32, K=48, predict=1,
         importance_rule=1, reuse=0),
    dict(H=257, W=383, cells=20, seed=5, num_levels=2, ratio_C=2, init_block=8, K=150, size_mode=1),
    dict(H=300, W=300, cells=30, seed=9, num_levels=1, init_block=16, K=300, size_mode=0),
    dict(H=512, W=512, cells=60, seed=3, num_levels=3, ratio_C=4, init_block=32, K=256, predict=1, final_grain=4),
    dict(H=640, W=512, cells=80, seed=4, num_levels=3, ratio_C=4, init_block=32, K=320, predict=1),
]


@pytest.mark.parametrize("case", MID, ids=[f"m{i}" for i in range(len(MID))])
def test_mid_size(case):
    c = dict(case)
    H, W, cells, seed = c.pop("H"), c.pop("W"), c.pop("cells"), c.pop("seed")
    rgb = synth.he_image(H, W, cells, seed).rgb
    assert_parity(rgb, **c)


def test_host_input_equals_device_input():
    rgb = synth.he_image(120, 160, 10, 2).rgb
    p = dict(K=40, init_block=8, num_levels=2, ratio_C=2, predict=1)
    a = gpu_run(rgb, device_input=True, **p)
    b = gpu_run(rgb, device_input=False, **p)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_stepwise_api_matches_oracle_after_every_stage():
    import torch

    import paper_1704_02083_gb300 as pkg
    rgb = synth.he_image(160, 224, 12, 8).rgb
    p = dict(num_levels=3, ratio_C=4, init_block=32, K=60, predict=1)
    o = oracle.Oracle(rgb, **p)
    o.seed()
    with pkg.Context(stream=torch.cuda.current_stream(), **p) as ctx:
        ctx.set_image(rgb)
        assert ctx.seed() == o.grid()["M"]
        for st in range(o.num_stages()):
            if st > 0:
                ctx.split()
                o.next_stage()
            np.testing.assert_array_equal(ctx.block_labels(), o.block_labels())
            sweeps, moves, merges = ctx.refine_stage(sync=True)
            o.refine_stage()
            c = o.counters()[st]
            assert (sweeps, moves, merges) == (c[2], c[5], c[7])
            np.testing.assert_array_equal(ctx.block_labels(), o.block_labels())
            s = ctx.stats()
            np.testing.assert_array_equal(s["n"], o.stats()[0][:, 0])
        with pytest.raises(pkg.RapidError) as e:
            ctx.split()
        assert e.value.status == pkg.RAPID_ESTATE


EDGE = [
    dict(H=1, W=1, K=1),
    dict(H=1, W=97, K=5, init_block=4),
    dict(H=83, W=1, K=5, init_block=4),
    dict(H=33, W=47, K=1000, init_block=8),          # K above the block count: clamped
    dict(H=40, W=40, K=4, init_block=1),             # single stage at full resolution
    dict(H=40, W=40, K=4, init_block=4, final_grain=8),   # final grain above the first block
    dict(H=64, W=64, K=16, init_block=64),           # one block at the first stage
    dict(H=50, W=70, K=9, num_levels=4, ratio_C=2, init_block=2, predict=1),  # init below f_1
]


@pytest.mark.parametrize("case", EDGE, ids=[f"e{i}" for i in range(len(EDGE))])
def test_edge_cases(case):
    c = dict(case)
    H, W = c.pop("H"), c.pop("W")
    rgb = synth.he_image(H, W, 3, H * 131 + W).rgb
    assert_parity(rgb, **c)


def test_flat_image_makes_no_move():
    rgb = synth.flat_image(256, 256)
    lab, st, cnt = assert_parity(rgb, K=16, init_block=16)
    assert cnt[:, 5].sum() == 0


def _golden(name):
    path = os.path.join(GOLDEN, f"{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"{path} not written")
    return json.load(open(path))


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


@pytest.mark.parametrize("name", ["he321x481_k200", "he4096_k4096_l3", "he321x481_k200_frontier",
                                  "he4096_k4096_l3_frontier"])
def test_full_size_against_golden(name):
    """Full-size workloads in the bench's launch configuration against the oracle's stored
    output (tests/golden, written by make_golden.py from the oracle alone)."""
    g = _golden(name)
    img = synth.workload_image(name)
    assert _sha(img.rgb) == g["image_sha256"], "generator output differs from the golden's"
    lab, st, y, imp, cnt = gpu_run(img.rgb, **g["params"])
    for yy, xx, v in g["samples"]:
        assert lab[yy, xx] == v
    assert cnt.tolist() == g["counters"]
    assert _sha(lab.astype("<i4")) == g["labels_sha256"]
    assert _sha(st.astype("<i8")) == g["stats_sha256"]
    assert _sha(y.astype("i1")) == g["y_sha256"]
    assert _sha(imp.astype("u1")) == g["important_sha256"]
