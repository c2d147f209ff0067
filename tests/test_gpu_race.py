"""The race check (rapid_set_race_check): every label write of a phase must be of a block of
the phase's class, written once, with no other write of the phase within distance 2 -- the
independence the 9-phase schedule rests on.  The check must find its scripted violations,
and none on real runs of both schedules (single images, a batch, the 321x481 workload),
whose results stay bit-exact against the oracle."""
import numpy as np
import pytest

from gpu_common import oracle_run
from paper_1704_02083_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def test_the_check_finds_scripted_violations():
    import paper_1704_02083_gb300 as pkg

    assert pkg.rapid_race_selftest() == [0, 2, 1]


CASES = [
    ("bsd321x481", lambda: synth.workload_image("he321x481_k200").rgb,
     dict(synth.WORKLOADS["he321x481_k200"]["params"])),
    ("he256_l3", lambda: synth.he_image(256, 256, 30, 21).rgb,
     dict(num_levels=3, ratio_C=4, init_block=32, K=64, size_mode=2, predict=1)),
    ("rand61x47", lambda: synth.random_image(61, 47, 8, levels=5),
     dict(num_levels=2, ratio_C=2, init_block=8, K=20, size_mode=2, predict=1, importance_rule=1)),
]


@pytest.mark.parametrize("schedule", [0, 1], ids=["sweeps", "queue"])
@pytest.mark.parametrize("name,img,params", CASES, ids=[c[0] for c in CASES])
def test_no_race_on_real_runs(name, img, params, schedule):
    import torch

    import paper_1704_02083_gb300 as pkg

    rgb = img()
    p = dict(params, schedule=schedule)
    with pkg.Context(stream=torch.cuda.current_stream(), **p) as ctx:
        ctx.set_race_check(True)
        ctx.set_image(torch.from_numpy(rgb).cuda()).run()
        lab = ctx.labels()
        moves = int(ctx.counters_array()[:, 5].sum())
        assert ctx.race_violations() == 0
    assert moves > 0
    np.testing.assert_array_equal(lab, oracle_run(rgb, **p)[0])


def test_no_race_in_a_batch():
    import torch

    import paper_1704_02083_gb300 as pkg

    imgs = [synth.he_image(96, 144, 6, 11).rgb, synth.random_image(37, 53, 12, levels=4),
            synth.he_image(70, 70, 4, 15).rgb]
    with pkg.Context(stream=torch.cuda.current_stream(), num_levels=2, ratio_C=4, init_block=16, size_mode=2,
                     predict=1) as ctx:
        ctx.set_race_check(True)
        ctx.set_images([torch.from_numpy(x).cuda() for x in imgs], [24, 9, 20])
        ctx.run()
        assert ctx.race_violations() == 0
