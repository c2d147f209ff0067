"""The oracle's superpixel features at the prediction point (the F in R^4 of Sec. 4.1:
absolute and comparative brightness, extra- and intra-region dissimilarity) and the linear
classifier of Eq. predict, pinned against:
  * a block-level restatement of the definitions from the full-resolution image and the
    label map alone (statistics recomputed, block sums from the pixels, pairs enumerated);
  * closed forms: a constant image, and uniform superpixels on a two-colour image;
  * theta = (3T, -3, 0, 0, 0), which must reproduce the integer brightness rule exactly."""
import math

import numpy as np
import pytest

import helpers
import oracle
from paper_1704_02083_gb300 import synth


def _to_prediction(o):
    """Step to the last level-1 stage; returns its block labels and side (the prediction
    grid), then enters level 2 (which runs the prediction)."""
    o.seed()
    o.refine_stage()
    stages = o.stages()
    while stages[o.grid()["stage"] + 1][0] < 2:
        o.next_stage()
        o.refine_stage()
    g = o.grid()
    bl = o.block_labels()
    o.next_stage()
    return bl, g["side"]


def _features_by_definition(rgb, bl, side, M):
    H, W = rgb.shape[:2]
    full = helpers.upsample(bl, side, H, W)
    S = helpers.stats_from_labels(rgb, full, M)  # N, R, G, B, X, Y
    N = [int(v) for v in S[:, 0]]
    C = [[int(S[k, 1 + c]) for c in range(3)] for k in range(M)]
    mean = [[C[k][c] / N[k] for c in range(3)] if N[k] else [0.0] * 3 for k in range(M)]
    sb, sd, si, npairs = [0] * M, [0] * M, [0] * M, [0] * M
    nby, nbx = bl.shape
    img = rgb.astype(np.int64)
    for by in range(nby):
        for bx in range(nbx):
            a = int(bl[by, bx])
            blk = img[by * side:min(by * side + side, H), bx * side:min(bx * side + side, W)]
            w = float(blk.shape[0] * blk.shape[1])
            cs = [int(blk[..., c].sum()) for c in range(3)]
            d = [cs[c] / w - mean[a][c] for c in range(3)]
            si[a] += int(w * (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * 65536.0)
            for qx, qy in ((bx + 1, by), (bx, by + 1)):
                if qx >= nbx or qy >= nby:
                    continue
                b = int(bl[qy, qx])
                if b == a:
                    continue
                sb[a] += (sum(C[b]) << 16) // (3 * N[b])
                sb[b] += (sum(C[a]) << 16) // (3 * N[a])
                npairs[a] += 1
                npairs[b] += 1
                e = [mean[a][c] - mean[b][c] for c in range(3)]
                dq = int(math.sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]) * 65536.0)
                sd[a] += dq
                sd[b] += dq
    F = np.zeros((M, 4))
    for k in range(M):
        if N[k] == 0:
            continue
        F[k, 0] = sum(C[k]) / (3 * N[k])
        if npairs[k]:
            F[k, 1] = F[k, 0] - (sb[k] / npairs[k]) / 65536.0
            F[k, 2] = (sd[k] / npairs[k]) / 65536.0
        F[k, 3] = math.sqrt((si[k] / 65536.0) / N[k])
    return F


CASES = [(40, 56, 12, 8, 2, 2, 3), (64, 48, 16, 16, 3, 2, 5), (33, 47, 9, 4, 2, 4, 7), (96, 80, 24, 16, 3, 4, 11)]


@pytest.mark.parametrize("H,W,K,ib,L,C,seed", CASES)
def test_features_match_their_definition(H, W, K, ib, L, C, seed):
    rgb = synth.he_image(H, W, 5, seed).rgb
    o = oracle.Oracle(rgb, K=K, init_block=ib, num_levels=L, ratio_C=C, predict=1)
    bl, side = _to_prediction(o)
    M = o.grid()["M"]
    got = o.features()
    want = _features_by_definition(rgb, bl, side, M)
    np.testing.assert_array_equal(got, want)
    assert (got[:, 2] > 0).sum() > 0 and (got[:, 3] > 0).sum() > 0


def test_constant_image_features():
    rgb = np.full((64, 64, 3), (90, 120, 150), np.uint8)
    o = oracle.Oracle(rgb, K=16, init_block=8, num_levels=2, ratio_C=2, predict=1)
    _to_prediction(o)
    F = o.features()
    np.testing.assert_array_equal(F[:, 0], np.full(F.shape[0], 120.0))
    np.testing.assert_array_equal(F[:, 1:], 0.0)


def test_two_colour_uniform_superpixels():
    """Superpixels that stay inside one colour: f4 = 0, f1 is the colour's brightness, and a
    superpixel touching the other colour has f3 = |A - B| times its share of pairs across."""
    H, W = 64, 64
    rgb = np.zeros((H, W, 3), np.uint8)
    rgb[:, :32] = (40, 60, 80)
    rgb[:, 32:] = (200, 180, 160)
    o = oracle.Oracle(rgb, K=16, init_block=16, num_levels=2, ratio_C=2, predict=1, max_sweeps=1)
    bl, side = _to_prediction(o)
    F = o.features()
    full = helpers.upsample(bl, side, H, W)
    dist = math.sqrt(160.0 ** 2 + 120.0 ** 2 + 80.0 ** 2)
    for k in np.unique(full):
        cols = np.unique(np.argwhere(full == k)[:, 1] < 32)
        assert len(cols) == 1  # the superpixel stays on one side
        left = bool(cols[0])
        assert F[k, 0] == (60.0 if left else 180.0)
        assert F[k, 3] == 0.0
        # pairs of k's blocks with other labels, and those that cross the colour edge
        pairs = cross = 0
        nby, nbx = bl.shape
        for by in range(nby):
            for bx in range(nbx):
                for qx, qy in ((bx + 1, by), (bx, by + 1), (bx - 1, by), (bx, by - 1)):
                    if not (0 <= qx < nbx and 0 <= qy < nby) or bl[by, bx] != k or bl[qy, qx] == k:
                        continue
                    pairs += 1
                    cross += (qx * side < 32) != (bx * side < 32)
        if pairs:
            assert abs(F[k, 2] - dist * cross / pairs) < 1e-4


def test_theta_reproduces_the_brightness_rule():
    """h = 3T - 3 f1 has the sign of 3 T N - (R + G + B): the same y, importance and run."""
    img = synth.he_image(128, 160, 10, 4)
    p = dict(K=60, init_block=16, num_levels=2, ratio_C=4, predict=1)
    a = oracle.Oracle(img.rgb, **p).run()
    b = oracle.Oracle(img.rgb, **p).set_classifier([3 * 150.0, -3.0, 0.0, 0.0, 0.0]).run()
    sa, ya, ia = a.stats()
    sb, yb, ib = b.stats()
    np.testing.assert_array_equal(ya, yb)
    np.testing.assert_array_equal(ia, ib)
    np.testing.assert_array_equal(a.labels(), b.labels())
    assert (ya == 1).any() and (ya == -1).any()


def test_classifier_sign_decides_the_class():
    """A constant h: theta_0 >= 0 makes every superpixel ROI (no boundary superpixel, no
    block refined after the prediction); theta_0 < 0 makes none ROI."""
    img = synth.he_image(96, 96, 8, 6)
    p = dict(K=36, init_block=16, num_levels=2, ratio_C=4, predict=1)
    for t0, cls in ((0.0, 1), (-1e-9, -1)):
        o = oracle.Oracle(img.rgb, **p).set_classifier([t0, 0.0, 0.0, 0.0, 0.0]).run()
        _, y, imp = o.stats()
        assert (y == cls).all() and not imp.any()
        assert o.counters()[o.num_stages() - 1, 3] == 0  # nothing eligible after the prediction


def test_generic_theta_weights_each_feature():
    """y from a generic theta is the sign of theta_0 + theta_1 f1 + ... + theta_4 f4 over the
    superpixel's own features (weights in feature order, summed left to right)."""
    img = synth.he_image(128, 128, 12, 9)
    p = dict(K=64, init_block=16, num_levels=2, ratio_C=4, predict=1)
    rng = np.random.default_rng(3)
    seen = 0
    for _ in range(6):
        t = rng.normal(0, 1, 5) * np.array([50.0, 0.3, 1.0, 0.5, 0.8])
        o = oracle.Oracle(img.rgb, **p).set_classifier(t)
        _to_prediction(o)
        F = o.features()
        _, y, _ = o.stats()
        live = F[:, 0] > 0
        h = (((t[0] + t[1] * F[:, 0]) + t[2] * F[:, 1]) + t[3] * F[:, 2]) + t[4] * F[:, 3]
        np.testing.assert_array_equal(y[live], np.where(h[live] >= 0, 1, -1))
        seen += int((y[live] == 1).any() and (y[live] == -1).any())
    assert seen >= 2
