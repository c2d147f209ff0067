"""Levels, stages, reuse (Eq. eq:mu) and prediction (Eq. predict, Eq. new_bound)."""
import numpy as np

import helpers
import oracle
from paper_1704_02083_gb300 import synth

P3 = dict(num_levels=3, ratio_C=4, init_block=32, K=48, predict=1, reuse=1)


def _img():
    return synth.he_image(200, 264, n_cells=14, seed=21).rgb


def test_stage_schedule():
    o = oracle.Oracle(_img(), **P3)
    assert o.stages() == [(1, 32), (1, 16), (2, 8), (2, 4), (3, 2), (3, 1)]
    o = oracle.Oracle(_img(), **{**P3, "final_grain": 4})
    assert o.stages() == [(1, 32), (1, 16), (2, 8), (2, 4)]
    o = oracle.Oracle(_img(), num_levels=1, init_block=16)
    assert o.stages() == [(1, 16), (1, 8), (1, 4), (1, 2), (1, 1)]
    o = oracle.Oracle(_img(), num_levels=2, ratio_C=2, init_block=4)
    assert o.stages() == [(1, 4), (1, 2), (2, 1)]


def test_pyramid_is_box_sums():
    rgb = _img()
    H, W = rgb.shape[:2]
    o = oracle.Oracle(rgb, **P3)
    for level, f in ((1, 16), (2, 4), (3, 1)):
        Wl, Hl, ff = o.level_dims(level)
        assert ff == f and Wl == -(-W // f) and Hl == -(-H // f)
        pyr = o.pyramid(level)
        pad = np.zeros((Hl * f, Wl * f, 6), np.int64)
        yy, xx = np.mgrid[0:H, 0:W]
        pad[:H, :W, 0] = 1
        pad[:H, :W, 1:4] = rgb
        pad[:H, :W, 4] = xx
        pad[:H, :W, 5] = yy
        ref = pad.reshape(Hl, f, Wl, f, 6).sum((1, 3))
        np.testing.assert_array_equal(pyr, ref)


def test_reuse_on_equals_recompute_each_level():
    """Carrying S across levels (RAPID) and recomputing it from each level (multi-scale
    CTFTPS) give identical results: with exact box sums Eq. eq:mu is exact."""
    rgb = _img()
    a = oracle.Oracle(rgb, **P3).run()
    b = oracle.Oracle(rgb, **{**P3, "reuse": 0}).run()
    np.testing.assert_array_equal(a.labels(), b.labels())
    np.testing.assert_array_equal(a.stats()[0], b.stats()[0])
    np.testing.assert_array_equal(a.counters(), b.counters())


def test_eq_mu_centroid_map():
    """Eq. eq:mu: a superpixel made of whole level-l pixels has, in level-(l+1) 1-based
    coordinates, centroid C*mu_l - (C-1)/2 where mu_l is its level-l 1-based centroid."""
    rng = np.random.default_rng(5)
    C = 4
    for _ in range(50):
        Hc, Wc = rng.integers(2, 9, 2)
        mask = rng.random((Hc, Wc)) < 0.5
        mask[rng.integers(Hc), rng.integers(Wc)] = True
        Y, X = np.nonzero(mask)
        mu_c = np.array([X.mean() + 1, Y.mean() + 1])
        fine = np.repeat(np.repeat(mask, C, 0), C, 1)
        y, x = np.nonzero(fine)
        mu_f = np.array([x.mean() + 1, y.mean() + 1])
        np.testing.assert_allclose(mu_f, C * mu_c - (C - 1) / 2, rtol=0, atol=1e-12)


def test_prediction_and_boundary_superpixels():
    """At level-2 entry: y_k = 1 iff 3 T N_k - (R_k + G_k + B_k) >= 0 (Eq. predict with the
    stand-in classifier); boundary superpixels are those 4-adjacent to the other class."""
    rgb = _img()
    H, W = rgb.shape[:2]
    o = oracle.Oracle(rgb, **P3)
    o.seed()
    o.refine_stage()
    o.next_stage()
    o.refine_stage()
    g = o.grid()
    lab1 = helpers.upsample(o.block_labels(), g["side"], H, W)
    s1, _, _ = o.stats()
    o.next_stage()  # enters level 2: prediction happens here
    s, y, imp = o.stats()
    np.testing.assert_array_equal(s, s1)
    live = s[:, 0] > 0
    h = 3 * 150 * s[:, 0] - s[:, 1:4].sum(1)
    np.testing.assert_array_equal(y[live], np.where(h[live] >= 0, 1, -1))
    exp = np.zeros(g["M"], bool)
    for A, B in ((lab1[:, :-1], lab1[:, 1:]), (lab1[:-1, :], lab1[1:, :])):
        d = (A != B) & (y[A] != y[B])
        exp[A[d]] = True
        exp[B[d]] = True
    np.testing.assert_array_equal(imp.astype(bool), exp)
    assert 0 < exp.sum() < live.sum()


def test_importance_prunes_work_at_later_levels():
    rgb = _img()
    on = oracle.Oracle(rgb, **P3).run().counters()
    off = oracle.Oracle(rgb, **{**P3, "predict": 0}).run().counters()
    assert (on[:2] == off[:2]).all()          # level 1 is identical
    assert on[2:, 3].sum() < off[2:, 3].sum()  # fewer eligible blocks later
    rule1 = oracle.Oracle(rgb, **{**P3, "importance_rule": 1}).run().counters()
    assert (rule1[:2] == off[:2]).all()
    assert rule1[2:, 3].sum() < off[2:, 3].sum()


def test_prediction_tie_is_roi():
    """Eq. predict: h >= 0 gives y = 1; a superpixel of mean brightness exactly T has h = 0."""
    H, W = 64, 128
    rgb = synth.two_colour_image(H, W, 64, left=(150, 150, 150), right=(200, 200, 200))
    o = oracle.Oracle(rgb, num_levels=2, ratio_C=4, init_block=16, K=2, predict=1)
    o.seed()
    o.refine_stage()
    while o.grid()["level"] < 2:
        o.next_stage()
    s, y, imp = o.stats()
    assert s[0, 1:4].sum() == 3 * 150 * s[0, 0]
    assert y.tolist() == [1, -1]
    assert imp.tolist() == [1, 1]
