"""The 64-tile batch workload at full size (251 Mpx, tiles of 512 to 4096 px a side), in
the bench's launch configuration: one context over all tiles, autotuned stage geometry,
CUDA graph capture and replay.  Every tile's labels, statistics, classes, importance and
counters must equal the oracle's record of that tile refined alone.  The records are
tests/golden/batch64_l3*.json, written by make_golden.py from the oracle only.  This file
is collected after every other GPU test because its run is the longest."""
import hashlib
import json
import os

import numpy as np
import pytest

from gpu_common import STAT_FIELDS
from paper_1704_02083_gb300 import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


@pytest.fixture(scope="module")
def tiles():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return synth.batch_workload("batch64_l3")  # the frontier variant refines the same tiles


@pytest.mark.parametrize("name", ["batch64_l3", "batch64_l3_frontier"])
def test_full_batch_against_golden(tiles, name):
    import torch

    import paper_1704_02083_gb300 as pkg

    path = os.path.join(GOLDEN, f"{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"{path} not written")
    g = json.load(open(path))
    imgs, K = tiles
    assert len(g["tiles"]) == len(imgs) == synth.BATCHES[name]["n"]
    for i, (rgb, k) in enumerate(zip(imgs, K)):
        t = g["tiles"][i]
        assert (t["tile"], t["H"], t["W"], t["K"]) == (i, rgb.shape[0], rgb.shape[1], k)
        assert _sha(rgb) == t["image_sha256"], f"tile {i}: generator output differs from the record's"
    stream = torch.cuda.Stream()  # a graph needs a non-default stream
    with torch.cuda.stream(stream):
        dev = [torch.from_numpy(x).cuda() for x in imgs]
        with pkg.Context(stream=stream, **g["params"]) as ctx:
            ctx.set_images(dev, K)
            ctx.autotune()
            ctx.set_graph(True)
            for rep in range(2):  # capture, then replay
                ctx.run()
                bad = []
                for i, t in enumerate(g["tiles"]):
                    lab = ctx.image_labels(i)
                    st = ctx.image_stats(i)
                    stats = np.stack([st[f] for f in STAT_FIELDS], 1)
                    checks = {
                        "samples": all(lab[y, x] == v for y, x, v in t["samples"]),
                        "counters": ctx.counters_array(i).tolist() == t["counters"],
                        "labels": _sha(lab.astype("<i4")) == t["labels_sha256"],
                        "stats": _sha(stats.astype("<i8")) == t["stats_sha256"],
                        "y": _sha(st["y"].astype("i1")) == t["y_sha256"],
                        "important": _sha(st["important"].astype("u1")) == t["important_sha256"],
                    }
                    bad += [(rep, i, k) for k, ok in checks.items() if not ok]
                assert not bad, f"{name}: (replay, tile, field) differing from the oracle: {bad[:12]}"
        del dev
