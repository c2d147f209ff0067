"""Host helpers of bench.py: the stage kernel's code hash that keys the committed DRAM
counters (comments and blank lines do not change it, code does), and the algorithmic
bytes of a stage launch under both schedules."""
import os
import shutil
import types

import bench

CSRC = os.path.join(bench.ROOT, "paper_1704_02083_gb300", "csrc")


def _copy(tmp_path):
    d = tmp_path / "csrc"
    shutil.copytree(CSRC, d)
    return str(d)


def test_code_hash_ignores_comments_but_not_code(tmp_path):
    d = _copy(tmp_path)
    h0 = bench.kernel_source_sha256(d)
    assert h0 == bench.kernel_source_sha256()
    p = os.path.join(d, "stage_impl.cuh")
    src = open(p).read()
    open(p, "w").write("// a new comment line\n\n" + src.replace("\n", "  // trailing note\n", 1))
    assert bench.kernel_source_sha256(d) == h0
    open(p, "w").write(src.replace("kMergeSet = 64", "kMergeSet = 32"))
    assert bench.kernel_source_sha256(d) != h0


def test_stage_alg_bytes_both_schedules():
    st = types.SimpleNamespace(block=1, level=3, sweeps=64, moves=1000, eligible=50000)
    lf = {1: 16, 2: 4, 3: 1}
    H = W = 4096
    nb = H * W
    assert bench.stage_alg_bytes(H, W, st, lf) == 4 * nb * 64 + 4 * 1000 + 3 * H * W
    assert bench.stage_alg_bytes(H, W, st, lf, True) == nb * 64 / 8 + 4 * 50000 + 4 * 1000 + 3 * H * W
    coarse = types.SimpleNamespace(block=32, level=1, sweeps=6, moves=10, eligible=100)
    nbc = (H // 32) * (W // 32)
    assert bench.stage_alg_bytes(H, W, coarse, lf) == 4 * nbc * 6 + 40 + 12 * (H // 16) * (W // 16)


def test_cpu_sample_keeps_the_workload_density():
    """The CPU legs time a sample with the workload's pixels per superpixel and per region;
    an image that fits the sample is sampled whole (the workload itself)."""
    import numpy as np

    from paper_1704_02083_gb300 import synth
    rgb, params, desc = bench.cpu_sample("he321x481_k200")
    w = synth.WORKLOADS["he321x481_k200"]
    assert rgb.shape == (w["H"], w["W"], 3) and params == w["params"]
    np.testing.assert_array_equal(rgb, synth.workload_image("he321x481_k200").rgb)
    assert desc.startswith("321x481 tile") and "K=200" in desc
    rgb, params, desc = bench.cpu_sample("he4096_k4096_l3")
    w = synth.WORKLOADS["he4096_k4096_l3"]
    assert rgb.shape == (bench.SAMPLE_SIDE, bench.SAMPLE_SIDE, 3)
    npx = bench.SAMPLE_SIDE ** 2
    assert npx / params["K"] == w["H"] * w["W"] / w["params"]["K"]
    assert f"{round(w['n_cells'] * npx / (w['H'] * w['W']))} regions" in desc
    rgb, params, _ = bench.cpu_sample("batch64_l3")
    assert params["K"] == npx // synth.BATCHES["batch64_l3"]["px_per_superpixel"]


class _OracleCtx:
    """Stands in for a context: each image's labels and statistics from the oracle."""

    def __init__(self, imgs, params_per_image):
        import numpy as np
        import oracle

        self.out = []
        for rgb, p in zip(imgs, params_per_image):
            o = oracle.Oracle(rgb, **p).run()
            s, y, imp = o.stats()
            st = np.zeros(s.shape[0], [(f, "<i8") for f in ("n", "sum_r", "sum_g", "sum_b", "sum_x", "sum_y",
                                                             "init_size")])
            for j, f in enumerate(st.dtype.names):
                st[f] = s[:, j]
            self.out.append((o.labels(), st))

    def image_labels(self, i):
        return self.out[i][0]

    def image_stats(self, i):
        return self.out[i][1]


def test_golden_parity_single_and_batch(tmp_path):
    import json
    import sys

    from paper_1704_02083_gb300 import synth
    sys.path.insert(0, os.path.join(bench.ROOT, "tests", "golden"))
    import make_golden

    w = synth.WORKLOADS["he321x481_k200"]
    img = synth.workload_image("he321x481_k200").rgb
    ctx = _OracleCtx([img], [w["params"]])
    assert bench.golden_parity("he321x481_k200", [img], ctx) == "bit-exact vs the oracle's golden hashes (labels, S)"
    ctx.out[0][0][5, 7] += 1
    assert bench.golden_parity("he321x481_k200", [img], ctx) == "MISMATCH vs the oracle's golden hashes"
    assert bench.golden_parity("no_such_workload", [img], ctx) is None
    # a batch record: one entry per tile
    imgs = [synth.he_image(40, 56, 4, 1).rgb, synth.he_image(33, 20, 3, 2).rgb]
    params = [dict(K=12, init_block=8), dict(K=5, init_block=4)]
    path = tmp_path / "b.json"
    path.write_text(json.dumps({"tiles": [make_golden.record(x, p) for x, p in zip(imgs, params)]}))
    ctx = _OracleCtx(imgs, params)
    assert bench.golden_parity("b", imgs, ctx, str(path)) == \
        "bit-exact vs the oracle's golden hashes (labels, S of all 2 tiles)"
    ctx.out[1][1]["sum_x"][0] += 1
    assert bench.golden_parity("b", imgs, ctx, str(path)) == "MISMATCH vs the oracle's golden hashes"
    assert bench.golden_parity("b", imgs[:1], ctx, str(path)) is None
