"""The two exact shortcuts of the stage kernel: single-precision decisions with a certified
error bound (binary64 when undecided) and skipping decisions whose inputs did not change
(skip_tiles: unchanged blocks under the sweep schedule, unqueued tiles under the queue one).
Both must leave labels, statistics and every oracle counter unchanged, and the
single-precision decisions must never disagree with binary64."""
import numpy as np
import pytest

from gpu_common import gpu_counters, gpu_run, oracle_run
from paper_1704_02083_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


CASES = [
    ("bsd", synth.workload_image("he321x481_k200").rgb, synth.WORKLOADS["he321x481_k200"]["params"]),
    ("l3", synth.he_image(512, 640, 60, 4).rgb,
     dict(num_levels=3, ratio_C=4, init_block=32, K=320, predict=1, size_mode=2)),
    ("rand", synth.random_image(96, 128, 5, levels=4), dict(K=40, init_block=8, size_mode=1)),
    ("flat-ish", synth.random_image(80, 80, 6, levels=2), dict(K=16, init_block=4, size_mode=0, lambda_pos0=0.0)),
]


@pytest.mark.parametrize("name,rgb,params", CASES, ids=[c[0] for c in CASES])
def test_shortcuts_change_nothing(name, rgb, params):
    ref = gpu_run(rgb, use_filter=0, skip_tiles=0, **params)
    for uf, st in ((1, 0), (0, 1), (1, 1)):
        got = gpu_run(rgb, use_filter=uf, skip_tiles=st, **params)
        for x, y in zip(got, ref):
            np.testing.assert_array_equal(x, y, err_msg=f"use_filter={uf} skip_tiles={st}")
    o = oracle_run(rgb, **params)
    np.testing.assert_array_equal(ref[0], o[0])
    np.testing.assert_array_equal(ref[4], o[4])


@pytest.mark.parametrize("name,rgb,params", CASES, ids=[c[0] for c in CASES])
def test_filter_never_disagrees_with_binary64(name, rgb, params):
    stages, _ = gpu_counters(rgb, verify_filter=1, **params)
    assert sum(s.filter_mismatches for s in stages) == 0
    evaluated = sum(s.evaluated for s in stages)
    fallbacks = sum(s.fp64_fallbacks for s in stages)
    assert evaluated > 0
    assert fallbacks <= evaluated
    if name != "flat-ish":  # exact ties are common there and go to binary64 by design
        assert fallbacks < 0.05 * evaluated, (fallbacks, evaluated)


EXTREMES = [
    ("lam_pos0_0", dict(lambda_pos0=0.0)),
    ("lam_pos0_1e6", dict(lambda_pos0=1e6)),
    ("lam_b_0", dict(lambda_b=0.0)),
    ("lam_b_1e4", dict(lambda_b=1e4)),
    ("both_large", dict(lambda_pos0=1e6, lambda_b=1e4)),
]


@pytest.mark.parametrize("name,extra", EXTREMES, ids=[e[0] for e in EXTREMES])
def test_filter_at_parameter_extremes(name, extra):
    """The certified single-precision decisions where float magnitudes and the bound's
    widening are most stressed: position weights of 0 and 10^6, boundary weights of 0 and
    10^4, and coarse blocks (initial block 512 on a 2048 x 1536 image, blocks of 2^18
    pixels): no disagreement with binary64, and the run equal to the binary64-only run."""
    rgb = synth.he_image(2048, 1536, 80, 12).rgb
    params = dict(num_levels=3, ratio_C=4, init_block=512, final_grain=8, K=48, size_mode=2, predict=1,
                  max_sweeps=24, **extra)
    stages, _ = gpu_counters(rgb, verify_filter=1, **params)
    assert sum(s.filter_mismatches for s in stages) == 0
    assert sum(s.evaluated for s in stages) > 0
    ref = gpu_run(rgb, use_filter=0, **params)
    got = gpu_run(rgb, use_filter=1, **params)
    for x, y in zip(got, ref):
        np.testing.assert_array_equal(x, y, err_msg=name)


def test_tiles_are_skipped_on_long_stages():
    img = synth.he_image(512, 640, 60, 4).rgb
    stages, _ = gpu_counters(img, num_levels=3, ratio_C=4, init_block=32, K=320, predict=1)
    last = stages[-1]
    assert last.tiles_skipped > 0 and last.tiles_scanned > 0


def _run_with_grids(rgb, grids, autotune=False, **params):
    import torch

    import paper_1704_02083_gb300 as pkg

    with pkg.Context(stream=torch.cuda.current_stream(), **params) as ctx:
        ctx.set_image(torch.from_numpy(np.ascontiguousarray(rgb)).cuda())
        chosen = ctx.autotune() if autotune else None
        if grids is not None:
            ctx.set_stage_grids(grids)
            ctx.set_stage_shapes([i % 6 for i in range(len(grids))][::-1])
        ctx.run()
        st = ctx.stats()
        return ctx.labels(), np.stack([st[f] for f in ("n", "sum_r", "sum_x")], 1), ctx.counters_array(), chosen


@pytest.mark.parametrize("name,rgb,params", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_launch_grid_changes_nothing(name, rgb, params):
    """Any number of CTAs per stage (one, odd counts, the full grid) and any tile shape give
    the same run."""
    ref = _run_with_grids(rgb, None, **params)
    for grids in ([1] * 8, [3, 1, 7, 2, 5, 152, 9, 4], [2 ** i for i in range(8)]):
        got = _run_with_grids(rgb, grids, **params)
        for x, y in zip(got[:3], ref[:3]):
            np.testing.assert_array_equal(x, y, err_msg=f"grids={grids}")


def test_autotune_picks_valid_grids_and_keeps_results():
    import torch

    rgb, params = CASES[1][1], CASES[1][2]
    ref = _run_with_grids(rgb, None, **params)
    lab, st, cnt, (grids, shapes) = _run_with_grids(rgb, None, autotune=True, **params)
    full = torch.cuda.get_device_properties(0).multi_processor_count
    assert len(grids) == len(shapes) == cnt.shape[0]
    assert all(1 <= g <= full for g in grids) and all(0 <= k < 6 for k in shapes)
    np.testing.assert_array_equal(lab, ref[0])
    np.testing.assert_array_equal(st, ref[1])
    np.testing.assert_array_equal(cnt, ref[2])


@pytest.mark.parametrize("schedule", [0, 1], ids=["sweeps", "queue"])
def test_cluster_launches_change_nothing(schedule):
    """A single image's grids of 2 to 16 CTAs run as one thread-block cluster (hardware
    cluster barriers in place of the grid barrier): every stage at cluster sizes 16, 12, 8
    and 2 with every tile shape equals the full-grid run and the oracle; a batch at the same
    small grids (cooperative launches) through a captured graph and its replay equals its
    full-grid run."""
    import torch

    import paper_1704_02083_gb300 as pkg

    for name, rgb, params in CASES[:3]:
        p = dict(params, schedule=schedule)
        ref = _run_with_grids(rgb, None, **p)
        for grids in ([16] * 8, [12, 16, 8, 16, 12, 8, 16, 2], [2] * 8):
            got = _run_with_grids(rgb, grids, **p)
            for x, y in zip(got[:3], ref[:3]):
                np.testing.assert_array_equal(x, y, err_msg=f"{name} grids={grids}")
        np.testing.assert_array_equal(ref[0], oracle_run(rgb, **p)[0])
    imgs = [CASES[0][1], CASES[2][1], synth.he_image(70, 90, 4, 15).rgb]
    params = dict(num_levels=2, ratio_C=4, init_block=16, size_mode=2, predict=1, schedule=schedule)
    K = [200, 40, 20]
    out = []
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for grids in (None, [16, 8, 16, 12, 16, 16, 16, 16]):
            with pkg.Context(stream=stream, **params) as ctx:
                ctx.set_graph(True)
                ctx.set_images([torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in imgs], K)
                if grids is not None:
                    ctx.set_stage_grids(grids)
                for rep in range(2):  # capture, then replay
                    ctx.run()
                    out.append([ctx.image_labels(i) for i in range(len(imgs))])
    for run in out[1:]:
        for a, b in zip(run, out[0]):
            np.testing.assert_array_equal(a, b)
