"""GPU batches (rapid_set_images): several images of different sizes refined together,
each stage one persistent launch over all of them.  Every image must come out exactly as
when it is refined alone: bit-exact labels and statistics against the CPU oracle run on
that image, and the same counters (including the implementation's own tile and merge-cache
counters) as a single-image GPU run."""
import numpy as np
import pytest

from gpu_common import STAT_FIELDS, oracle_run
from paper_1704_02083_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _batch_images():
    """Uneven sizes (ragged against every block side), textures and a flat image that
    converges at once while the others keep sweeping."""
    imgs = [
        synth.he_image(96, 144, 6, 11).rgb,
        synth.random_image(37, 53, 12, levels=4),
        synth.he_image(128, 64, 5, 13).rgb,
        synth.random_image(1, 20, 14, levels=256),
        np.full((64, 64, 3), 200, np.uint8),
        synth.he_image(70, 70, 4, 15).rgb,
        synth.random_image(17, 5, 16, levels=2),
    ]
    K = [24, 9, 16, 3, 16, 20, 2]
    return imgs, K


def _run_batch(imgs, K, device_input=True, graph=False, **params):
    import torch

    import paper_1704_02083_gb300 as pkg

    stream = torch.cuda.Stream() if graph else torch.cuda.current_stream()
    out = []
    with torch.cuda.stream(stream):
        with pkg.Context(stream=stream, **params) as ctx:
            if graph:
                ctx.set_graph(True)
            src = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in imgs] if device_input else imgs
            ctx.set_images(src, K)
            for _ in range(2 if graph else 1):  # graph mode: capture, then replay
                ctx.run()
            for i in range(len(imgs)):
                st = ctx.image_stats(i)
                c = ctx.counters(i)
                out.append(dict(labels=ctx.image_labels(i), stats=np.stack([st[f] for f in STAT_FIELDS], 1),
                                y=st["y"].astype(np.int8), imp=st["important"].astype(np.uint8),
                                cnt=ctx.counters_array(i), full=[c.stage[s] for s in range(c.num_stages)]))
    return out


PARAMS = [
    dict(num_levels=2, ratio_C=4, init_block=16, size_mode=2, predict=1),
    dict(num_levels=1, init_block=8, size_mode=2, final_grain=2),
    dict(num_levels=3, ratio_C=2, init_block=8, size_mode=1, predict=1, importance_rule=1, reuse=0),
]


@pytest.mark.parametrize("params", PARAMS, ids=["l2_predict", "l1_grain2", "l3_rule1_noreuse"])
def test_batch_matches_oracle_per_image(params):
    imgs, K = _batch_images()
    res = _run_batch(imgs, K, **params)
    for i, (rgb, k) in enumerate(zip(imgs, K)):
        rlab, rst, ry, rimp, rcnt = oracle_run(rgb, K=k, **params)
        r = res[i]
        assert r["labels"].shape == rlab.shape
        diff = np.argwhere(r["labels"] != rlab)
        assert diff.size == 0, f"image {i}: {len(diff)} labels differ, first at {diff[:3].tolist()}"
        np.testing.assert_array_equal(r["stats"], rst, err_msg=f"image {i}")
        if params.get("predict", 0):
            np.testing.assert_array_equal(r["y"], ry, err_msg=f"image {i}")
            np.testing.assert_array_equal(r["imp"], rimp, err_msg=f"image {i}")
        np.testing.assert_array_equal(r["cnt"], rcnt, err_msg=f"image {i}")


def test_batch_equals_single_runs_including_fast_path_counters():
    import torch

    import paper_1704_02083_gb300 as pkg

    imgs, K = _batch_images()
    params = PARAMS[0]
    res = _run_batch(imgs, K, **params)
    fields = ("sweeps", "eligible", "evaluated", "moves", "merge_requests", "merges", "fp64_fallbacks",
              "tiles_scanned", "tiles_skipped", "merge_searches", "merge_cache_hits")
    for i, (rgb, k) in enumerate(zip(imgs, K)):
        with pkg.Context(stream=torch.cuda.current_stream(), K=k, **params) as ctx:
            ctx.set_image(torch.from_numpy(np.ascontiguousarray(rgb)).cuda()).run()
            lab = ctx.labels()
            c = ctx.counters()
            single = [c.stage[s] for s in range(c.num_stages)]
        np.testing.assert_array_equal(res[i]["labels"], lab)
        for s, (a, b) in enumerate(zip(res[i]["full"], single)):
            for f in fields:
                assert getattr(a, f) == getattr(b, f), f"image {i} stage {s} {f}"


def test_host_input_and_graph_replay_give_the_same_batch():
    imgs, K = _batch_images()
    params = PARAMS[0]
    ref = _run_batch(imgs, K, **params)
    for variant in (dict(device_input=False), dict(graph=True)):
        res = _run_batch(imgs, K, **variant, **params)
        for i in range(len(imgs)):
            np.testing.assert_array_equal(res[i]["labels"], ref[i]["labels"])
            np.testing.assert_array_equal(res[i]["stats"], ref[i]["stats"])
            np.testing.assert_array_equal(res[i]["cnt"], ref[i]["cnt"])


def test_batch_limits():
    import torch

    import paper_1704_02083_gb300 as pkg

    small = [np.zeros((4, 4, 3), np.uint8)] * (pkg.RAPID_MAX_BATCH + 1)
    with pkg.Context(stream=torch.cuda.current_stream(), K=1, init_block=2) as ctx:
        with pytest.raises(pkg.RapidError) as e:
            ctx.set_images(small)
        assert e.value.status == pkg.RAPID_ERANGE
        with pytest.raises(pkg.RapidError) as e:
            pkg.rapid_set_images(ctx.h, [], [], [], [], None, 0)
        assert e.value.status == pkg.RAPID_EINVAL
        ctx.set_images(small[:pkg.RAPID_MAX_BATCH]).run()
        assert ctx.image_labels(pkg.RAPID_MAX_BATCH - 1).shape == (4, 4)
        out = np.zeros((4, 4), np.int32)
        with pytest.raises(pkg.RapidError) as e:
            pkg.rapid_read_image_labels(ctx.h, pkg.RAPID_MAX_BATCH, out.ctypes.data, 16, 0)
        assert e.value.status == pkg.RAPID_EINVAL
