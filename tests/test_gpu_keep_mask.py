"""GPU parity of the pruned sweeps (the machinery the learned scorer drives), through the C
ABI: with the same seeded keep masks given to the library (rapid_set_keep_mask) and to the
oracle (orc_set_keep_mask), labels, statistics and every per-stage counter are bit-exact,
for single images, a batch (per image against the oracle) and a captured graph's replay.
The masks are inputs, drawn here: Bernoulli masks at several keep rates, masks for some
stages only, and a mask that keeps nothing."""
import zlib

import numpy as np
import pytest

import oracle
from gpu_common import STAT_FIELDS
from paper_1704_02083_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _grids(H, W, params):
    o = oracle.Oracle(np.zeros((H, W, 3), np.uint8), **{k: v for k, v in params.items() if k in oracle.DEFAULTS})
    return [(-(-H // side), -(-W // side)) for _, side in o.stages()]


def _masks(H, W, params, seed, rate, stages=None):
    """One mask per stage (None where `stages` leaves the stage unpruned)."""
    rng = np.random.default_rng(seed)
    out = []
    for s, g in enumerate(_grids(H, W, params)):
        m = (rng.random(g) < rate).astype(np.uint8)
        out.append(m if stages is None or s in stages else None)
    return out


def _oracle(rgb, masks, params, K=None):
    p = {k: v for k, v in params.items() if k in oracle.DEFAULTS}
    if K is not None:
        p["K"] = K
    o = oracle.Oracle(rgb, **p)
    for s, m in enumerate(masks):
        if m is not None:
            o.set_keep_mask(s, m)
    o.run()
    s, y, imp = o.stats()
    return o.labels(), s, o.counters()


def _gpu(rgb, masks, params):
    import torch

    import paper_1704_02083_gb300 as pkg

    with pkg.Context(stream=torch.cuda.current_stream(), **params) as ctx:
        ctx.set_image(torch.from_numpy(np.ascontiguousarray(rgb)).cuda())
        for s, m in enumerate(masks):
            if m is not None:
                ctx.set_keep_mask(0, s, m)
        ctx.run()
        st = ctx.stats()
        return ctx.labels(), np.stack([st[f] for f in STAT_FIELDS], 1), ctx.counters_array()


def _same(got, want, what):
    lab, st, cnt = got
    rlab, rst, rcnt = want
    diff = np.argwhere(lab != rlab)
    assert diff.size == 0, f"{what}: {len(diff)} labels differ, first at {diff[:3].tolist()}"
    np.testing.assert_array_equal(st, rst, err_msg=what)
    np.testing.assert_array_equal(cnt, rcnt, err_msg=what)


CASES = [
    ("he96x144_l2", lambda: synth.he_image(96, 144, 6, 11).rgb,
     dict(num_levels=2, ratio_C=4, init_block=16, K=24, size_mode=2, predict=1)),
    ("rand37x53_l1", lambda: synth.random_image(37, 53, 12, levels=4),
     dict(num_levels=1, init_block=8, K=9, size_mode=2, final_grain=1)),
    ("he128x64_l3_rule1", lambda: synth.he_image(128, 64, 5, 13).rgb,
     dict(num_levels=3, ratio_C=2, init_block=8, K=16, size_mode=1, predict=1, importance_rule=1, reuse=0)),
    ("bsd321x481", lambda: synth.workload_image("he321x481_k200").rgb,
     dict(synth.WORKLOADS["he321x481_k200"]["params"])),
]


@pytest.mark.parametrize("rate", [0.0, 0.3, 0.7, 1.0])
@pytest.mark.parametrize("name,img,params", CASES, ids=[c[0] for c in CASES])
def test_pruned_sweeps_match_the_oracle(name, img, params, rate):
    rgb = img()
    H, W = rgb.shape[:2]
    masks = _masks(H, W, params, seed=zlib.crc32(f"{name}:{rate}".encode()) % 1000, rate=rate)
    _same(_gpu(rgb, masks, params), _oracle(rgb, masks, params), f"{name} rate {rate}")


@pytest.mark.parametrize("name,img,params", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_masks_on_some_stages_only(name, img, params):
    rgb = img()
    H, W = rgb.shape[:2]
    n = len(_grids(H, W, params))
    masks = _masks(H, W, params, seed=7, rate=0.5, stages=set(range(0, n, 2)))
    _same(_gpu(rgb, masks, params), _oracle(rgb, masks, params), name)


def test_batch_with_masks_matches_the_oracle_per_image():
    """Three images in one context: masks for every stage of the first, for some stages of
    the second, none for the third (which then keeps every block at the pruned stages),
    through a captured graph and its replay."""
    import torch

    import paper_1704_02083_gb300 as pkg

    params = dict(num_levels=2, ratio_C=4, init_block=16, size_mode=2, predict=1)
    imgs = [synth.he_image(96, 144, 6, 11).rgb, synth.random_image(37, 53, 12, levels=4),
            synth.he_image(70, 70, 4, 15).rgb]
    K = [24, 9, 20]
    n = len(_grids(96, 144, params))
    masks = [_masks(*x.shape[:2], params, seed=20 + i, rate=0.5, stages=None if i == 0 else {1})
             for i, x in enumerate(imgs[:2])]
    pruned_stages = {s for s in range(n) if masks[0][s] is not None or masks[1][s] is not None}
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with pkg.Context(stream=stream, **params) as ctx:
            ctx.set_graph(True)
            ctx.set_images([torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in imgs], K)
            for i in range(2):
                for s, m in enumerate(masks[i]):
                    if m is not None:
                        ctx.set_keep_mask(i, s, m)
            for rep in range(2):  # capture, then replay
                ctx.run()
                for i, x in enumerate(imgs):
                    st = ctx.image_stats(i)
                    got = (ctx.image_labels(i), np.stack([st[f] for f in STAT_FIELDS], 1), ctx.counters_array(i))
                    # a stage is pruned for every image once any image has a mask for it; an
                    # image without a mask there keeps every block
                    given = masks[i] if i < 2 else [None] * n
                    mi = [given[s] if given[s] is not None else (np.ones(g, np.uint8) if s in pruned_stages else None)
                          for s, g in enumerate(_grids(*x.shape[:2], params))]
                    _same(got, _oracle(x, mi, params, K=K[i]), f"image {i} run {rep}")


def test_keep_mask_errors():
    import torch

    import paper_1704_02083_gb300 as pkg

    rgb = synth.he_image(64, 64, 4, 3).rgb
    params = dict(num_levels=1, init_block=8, K=9)
    nby, nbx = _grids(64, 64, params)[0]
    with pkg.Context(stream=torch.cuda.current_stream(), **params) as ctx:
        with pytest.raises(pkg.RapidError):  # before any image
            ctx.set_keep_mask(0, 0, np.ones((nby, nbx), np.uint8))
        ctx.set_image(torch.from_numpy(rgb).cuda())
        for i, s, shape in ((0, 0, (nby, nbx + 1)), (1, 0, (nby, nbx)), (0, 99, (nby, nbx)), (-1, 0, (nby, nbx))):
            with pytest.raises(pkg.RapidError):
                ctx.set_keep_mask(i, s, np.ones(shape, np.uint8))
        ctx.set_keep_mask(0, 0, np.zeros((nby, nbx), np.uint8))
        with pytest.raises(pkg.RapidError):  # one source of masks at a time
            ctx.set_scorer(np.zeros(3777, np.float32), 0.5)
        ctx.set_keep_mask(-1, -1, None)
        ctx.run()
        plain = ctx.labels()
    with pkg.Context(stream=torch.cuda.current_stream(), schedule=1, **params) as ctx:
        ctx.set_image(torch.from_numpy(rgb).cuda())
        with pytest.raises(pkg.RapidError):  # pruned sweeps belong to the sweep schedule
            ctx.set_keep_mask(0, 0, np.ones((nby, nbx), np.uint8))
    o = oracle.Oracle(rgb, **params).run()
    np.testing.assert_array_equal(plain, o.labels())  # cleared masks: the plain run
