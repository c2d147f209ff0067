"""GPU parity of the superpixel features (the F in R^4 of Sec. 4.1) and of Eq. predict with
a linear classifier on them: features, y, importance and the whole refinement after the
prediction equal the CPU oracle's bit for bit, for single images, batches and graph
replays; theta = (3T, -3, 0, 0, 0) reproduces the brightness stand-in."""
import numpy as np
import pytest

import oracle
from gpu_common import STAT_FIELDS, assert_parity, gpu_run
from paper_1704_02083_gb300 import synth
from test_gpu_parity import TINY

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _theta(seed):
    rng = np.random.default_rng(seed)
    t = rng.normal(0, 1, 5) * np.array([60.0, 0.4, 1.0, 0.5, 0.8])
    t[1] = -abs(t[1])
    return t


def _oracle_features(rgb, theta, **p):
    o = oracle.Oracle(rgb, **p).set_classifier(theta).run()
    return o.features(), o.stats()[1]


MID = [
    (synth.he_image(200, 264, 14, 21).rgb, dict(num_levels=3, ratio_C=4, init_block=32, K=48, predict=1)),
    (synth.he_image(257, 383, 20, 5).rgb, dict(num_levels=2, ratio_C=2, init_block=8, K=150, predict=1, size_mode=1)),
    (synth.he_image(512, 512, 60, 3).rgb, dict(num_levels=3, ratio_C=4, init_block=32, K=256, predict=1)),
    (synth.random_image(97, 131, 4, levels=4), dict(num_levels=2, ratio_C=4, init_block=8, K=30, predict=1,
                                                    importance_rule=1)),
]


@pytest.mark.parametrize("i", range(len(MID)))
def test_features_and_run_match_oracle(i):
    import torch

    import paper_1704_02083_gb300 as pkg

    rgb, p = MID[i]
    for seed in (i, 10 + i):
        theta = _theta(seed)
        with pkg.Context(stream=torch.cuda.current_stream(), **p) as ctx:
            ctx.set_classifier(theta)
            ctx.set_image(torch.from_numpy(np.ascontiguousarray(rgb)).cuda()).run()
            F = ctx.features()
            y = ctx.stats()["y"].astype(np.int8)
        rF, ry = _oracle_features(rgb, theta, **p)
        np.testing.assert_array_equal(F, rF)
        np.testing.assert_array_equal(y, ry)
        assert_parity(rgb, theta=theta, **p)


@pytest.mark.parametrize("case", [c for c in TINY if c["predict"] and c["num_levels"] > 1],
                         ids=lambda c: f"{c['H']}x{c['W']}s{c['seed']}")
def test_tiny_random_with_classifier(case):
    c = dict(case)
    H, W, seed, levels = c.pop("H"), c.pop("W"), c.pop("seed"), c.pop("levels")
    rgb = synth.random_image(H, W, seed, levels=levels) if seed % 2 else synth.he_image(H, W, 4, seed).rgb
    assert_parity(rgb, theta=_theta(seed), **c)


def test_standin_theta_equals_the_brightness_rule():
    img = synth.he_image(256, 320, 30, 12)
    p = dict(num_levels=3, ratio_C=4, init_block=32, K=120, predict=1)
    a = gpu_run(img.rgb, **p)
    b = gpu_run(img.rgb, theta=[3 * 150.0, -3.0, 0.0, 0.0, 0.0], **p)
    for x, z in zip(a, b):
        np.testing.assert_array_equal(x, z)


def test_batch_and_graph_replay_match_oracle():
    import torch

    import paper_1704_02083_gb300 as pkg

    imgs = [synth.he_image(96, 144, 6, 11).rgb, synth.he_image(128, 64, 5, 13).rgb,
            synth.random_image(70, 90, 15, levels=4)]
    K = [24, 16, 20]
    p = dict(num_levels=2, ratio_C=4, init_block=16, size_mode=2, predict=1)
    theta = _theta(5)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with pkg.Context(stream=stream, **p) as ctx:
            ctx.set_classifier(theta)
            ctx.set_graph(True)
            ctx.set_images([torch.from_numpy(x).cuda() for x in imgs], K)
            for rep in range(2):
                ctx.run()
                for i, (rgb, k) in enumerate(zip(imgs, K)):
                    o = oracle.Oracle(rgb, K=k, **p).set_classifier(theta).run()
                    np.testing.assert_array_equal(ctx.features(i), o.features(), err_msg=f"image {i} rep {rep}")
                    np.testing.assert_array_equal(ctx.image_labels(i), o.labels())
                    st = ctx.image_stats(i)
                    np.testing.assert_array_equal(st["y"].astype(np.int8), o.stats()[1])
                    np.testing.assert_array_equal(np.stack([st[f] for f in STAT_FIELDS], 1), o.stats()[0])


def test_errors():
    import torch

    import paper_1704_02083_gb300 as pkg

    with pkg.Context(stream=torch.cuda.current_stream(), K=8, predict=1, num_levels=2) as ctx:
        ctx.set_image(torch.zeros((32, 32, 3), dtype=torch.uint8, device="cuda"))
        with pytest.raises(pkg.RapidError) as e:
            ctx.features()
        assert e.value.status == pkg.RAPID_ESTATE
        with pytest.raises(pkg.RapidError) as e:
            ctx.set_classifier([0.0, float("nan"), 0.0, 0.0, 0.0])
        assert e.value.status == pkg.RAPID_EINVAL
