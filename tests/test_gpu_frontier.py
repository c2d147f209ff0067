"""GPU parity of the frontier schedule (schedule 1: the boundary queue of Sec. 2.1 as one
flag per block; a phase pops the queued blocks of its class, a move or an accepted merge
queues the 4-neighbours).  Labels, statistics and the oracle's counters of the CUDA path,
called through the C ABI, equal the CPU oracle's (schedule 1) bit for bit, for every tile
shape and launch grid of the stage kernel (the queue is kept per evaluation tile), in
batches, through the graph and no-allocation entry points."""
import numpy as np
import pytest

from gpu_common import STAT_FIELDS, assert_parity, gpu_run, oracle_run
from paper_1704_02083_gb300 import synth
from test_gpu_parity import EDGE, MID, TINY

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("case", TINY, ids=[f"t{i}" for i in range(len(TINY))])
def test_tiny_random(case):
    c = dict(case)
    H, W, seed, levels = c.pop("H"), c.pop("W"), c.pop("seed"), c.pop("levels")
    rgb = synth.random_image(H, W, seed, levels=levels) if seed % 2 else synth.he_image(H, W, 4, seed).rgb
    assert_parity(rgb, schedule=1, **c)


@pytest.mark.parametrize("case", MID, ids=[f"m{i}" for i in range(len(MID))])
def test_mid_size(case):
    c = dict(case)
    H, W, cells, seed = c.pop("H"), c.pop("W"), c.pop("cells"), c.pop("seed")
    rgb = synth.he_image(H, W, cells, seed).rgb
    lab, st, cnt = assert_parity(rgb, schedule=1, **c)
    assert cnt[:, 5].sum() > 0


@pytest.mark.parametrize("case", EDGE, ids=[f"e{i}" for i in range(len(EDGE))])
def test_edge_cases(case):
    c = dict(case)
    H, W = c.pop("H"), c.pop("W")
    rgb = synth.he_image(H, W, 3, H * 131 + W).rgb
    assert_parity(rgb, schedule=1, **c)


def _run_shapes(rgb, shape, grids, **params):
    import torch

    import paper_1704_02083_gb300 as pkg

    with pkg.Context(stream=torch.cuda.current_stream(), schedule=1, **params) as ctx:
        ctx.set_image(torch.from_numpy(np.ascontiguousarray(rgb)).cuda())
        ctx.set_stage_shapes([shape] * 16)
        if grids is not None:
            ctx.set_stage_grids((grids * 16)[:16])
        ctx.run()
        st = ctx.stats()
        return ctx.labels(), np.stack([st[f] for f in STAT_FIELDS], 1), ctx.counters_array()


SHAPE_CASES = [
    ("l3", synth.he_image(300, 420, 30, 4).rgb, dict(num_levels=3, ratio_C=4, init_block=32, K=160, predict=1)),
    ("rand", synth.random_image(150, 97, 5, levels=4), dict(K=40, init_block=8, size_mode=2)),
]


@pytest.mark.parametrize("name,rgb,params", SHAPE_CASES, ids=[c[0] for c in SHAPE_CASES])
def test_every_tile_shape_and_grid_gives_the_oracle_run(name, rgb, params):
    """The queue flags live per (tile, phase class): pushes across tile edges and ragged
    tiles must land on the block the oracle queues, whatever the shape and grid."""
    rlab, rst, _, _, rcnt = oracle_run(rgb, schedule=1, **params)
    for shape in range(6):
        for grids in (None, [1], [7, 3, 152]):
            lab, st, cnt = _run_shapes(rgb, shape, grids, **params)
            tag = f"shape {shape} grids {grids}"
            np.testing.assert_array_equal(lab, rlab, err_msg=tag)
            np.testing.assert_array_equal(st, rst, err_msg=tag)
            np.testing.assert_array_equal(cnt, rcnt, err_msg=tag)


def test_frontier_evaluates_fewer_blocks_than_sweeps():
    img = synth.he_image(512, 640, 60, 4).rgb
    p = dict(num_levels=3, ratio_C=4, init_block=32, K=320, predict=1)
    sweep = gpu_run(img, **p)[4]
    front = gpu_run(img, schedule=1, **p)[4]
    assert front[:, 3].sum() < 0.5 * sweep[:, 3].sum()  # eligible evaluations


def test_batch_matches_oracle_per_image():
    import torch

    import paper_1704_02083_gb300 as pkg

    imgs = [synth.he_image(96, 144, 6, 11).rgb, synth.random_image(37, 53, 12, levels=4),
            synth.he_image(128, 64, 5, 13).rgb, np.full((64, 64, 3), 200, np.uint8),
            synth.random_image(17, 5, 16, levels=2)]
    K = [24, 9, 16, 16, 2]
    params = dict(num_levels=2, ratio_C=4, init_block=16, size_mode=2, predict=1, schedule=1)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with pkg.Context(stream=stream, **params) as ctx:
            ctx.set_graph(True)
            ctx.set_images([torch.from_numpy(x).cuda() for x in imgs], K)
            for rep in range(2):  # capture, then replay: every launch starts with a full queue
                ctx.run()
                for i, (rgb, k) in enumerate(zip(imgs, K)):
                    rlab, rst, _, _, rcnt = oracle_run(rgb, K=k, **params)
                    st = ctx.image_stats(i)
                    np.testing.assert_array_equal(ctx.image_labels(i), rlab, err_msg=f"image {i} rep {rep}")
                    np.testing.assert_array_equal(np.stack([st[f] for f in STAT_FIELDS], 1), rst)
                    np.testing.assert_array_equal(ctx.counters_array(i), rcnt)


def test_scorer_is_refused_with_the_frontier_schedule():
    import torch

    import paper_1704_02083_gb300 as pkg

    with pkg.Context(stream=torch.cuda.current_stream(), K=8, schedule=1) as ctx:
        with pytest.raises(pkg.RapidError) as e:
            ctx.set_scorer(np.zeros(pkg.RAPID_SCORER_PARAMS, np.float32), 0.5)
        assert e.value.status == pkg.RAPID_EINVAL
