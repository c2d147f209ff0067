"""Closed-form special cases of the oracle (results fixed by the mathematics alone)."""
import numpy as np
import pytest

import helpers
import oracle
from paper_1704_02083_gb300 import synth


def test_constant_image_aligned_grid_makes_no_move():
    """Flat colour, grid cells aligned with the blocks: every block is nearer its own cell's
    centroid and any move lengthens the boundary, so no stage moves anything."""
    rgb = synth.flat_image(256, 256)
    for size_mode in (0, 2):
        o = oracle.Oracle(rgb, K=16, init_block=16, size_mode=size_mode).run()
        c = o.counters()
        assert c[:, 5].sum() == 0 and c[:, 7].sum() == 0
        assert (c[:, 2] == 1).all()
        lab = o.labels()
        expect = (np.arange(256)[:, None] // 64) * 4 + (np.arange(256)[None, :] // 64)
        np.testing.assert_array_equal(lab, expect)


@pytest.mark.parametrize("x0", [77, 70, 90, 65])
def test_two_colour_split_recovered_exactly(x0):
    """Two colours split at a column that is not block aligned, two superpixels, no
    position term: the refinement lands exactly on the colour edge."""
    H, W = 64, 128
    rgb = synth.two_colour_image(H, W, x0)
    o = oracle.Oracle(rgb, K=2, init_block=16, lambda_pos0=0.0, lambda_b=1.0, size_mode=2).run()
    assert o.grid()["M"] == 2
    lab = o.labels()
    expect = np.where(np.arange(W)[None, :] < x0, 0, 1) * np.ones((H, 1), np.int64)
    np.testing.assert_array_equal(lab, expect)


def test_single_pixel_and_single_superpixel():
    o = oracle.Oracle(np.zeros((1, 1, 3), np.uint8), K=1, init_block=16).run()
    assert o.counters()[:, 5].sum() == 0
    assert o.labels().tolist() == [[0]]
    rgb = synth.random_image(40, 56, seed=3)
    o = oracle.Oracle(rgb, K=1, init_block=8).run()
    assert o.grid()["M"] == 1
    assert o.counters()[:, 5].sum() == 0
    s, _, _ = o.stats()
    assert s[0, 0] == 40 * 56 and s[0, 6] == 40 * 56
    assert s[0, 4] == 56 * 55 // 2 * 40 and s[0, 5] == 40 * 39 // 2 * 56


def test_no_size_term_never_requests_merges():
    rgb = synth.he_image(64, 96, 6, seed=4).rgb
    o = oracle.Oracle(rgb, K=30, init_block=8, size_mode=0).run()
    c = o.counters()
    assert c[:, 6].sum() == 0 and c[:, 7].sum() == 0


def test_seed_grid_counts():
    """Regular seeding (Algorithm RAPID): gx = round(sqrt(K W / H)), gy = round(K / gx)."""
    o = oracle.Oracle(synth.flat_image(321, 481), K=200, init_block=16)
    o.seed()
    assert o.grid()["M"] == 17 * 12
    o = oracle.Oracle(synth.flat_image(64, 64), K=4096, init_block=32)  # clamped to 2x2 blocks
    o.seed()
    assert o.grid()["M"] == 4


@pytest.mark.parametrize("seed", [0, 3, 5])
def test_pixel_replicated_image_refines_to_replicated_labels(seed):
    """lambda_pos per unit of initial superpixel area: replicating every pixel 2 x 2, with
    blocks twice as large and no boundary term, multiplies the colour part of every energy
    difference of Eq. equa:energy1 by 4 and its position part by 16 (positions double, Eq.
    eq:mu; the sub-pixel offsets add a label-independent constant), so only lambda_pos =
    lambda_pos0 M / (H W), which falls by 4, keeps every decision, move and merge the same.  Pins the position weight's scaling, the position sums and the
    merge cost's position term."""
    for rgb, K, b in ((synth.he_image(48, 64, 6, seed).rgb, 12, 8),
                      (synth.random_image(20, 28, seed, levels=4), 6, 4)):
        big = np.repeat(np.repeat(rgb, 2, 0), 2, 1)
        p = dict(K=K, final_grain=1, lambda_b=0.0, lambda_pos0=400.0, size_mode=2)
        o1 = oracle.Oracle(rgb, init_block=b, **p).run()
        o2 = oracle.Oracle(big, init_block=2 * b, **{**p, "final_grain": 2}).run()
        np.testing.assert_array_equal(o2.labels(), np.repeat(np.repeat(o1.labels(), 2, 0), 2, 1))
        c1, c2 = o1.counters(), o2.counters()
        np.testing.assert_array_equal(c1[:, 2:], c2[:, 2:])
        assert c1[:, 5].sum() > 50
        assert o2.lambda_pos() * 4 == o1.lambda_pos()
