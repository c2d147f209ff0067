"""The seeded input generator holds to the recipe its docstring states: deterministic per
seed, the stated class shares, noise law and nucleus placement, the batch tile sizes and
the slide's fold coverage."""
import numpy as np
import pytest

from paper_1704_02083_gb300 import synth


def test_same_seed_same_bytes_other_seed_other_bytes():
    a = synth.he_image(96, 128, 12, seed=4)
    b = synth.he_image(96, 128, 12, seed=4)
    c = synth.he_image(96, 128, 12, seed=5)
    assert np.array_equal(a.rgb, b.rgb) and np.array_equal(a.regions, b.regions) and np.array_equal(a.roi, b.roi)
    assert not np.array_equal(a.rgb, c.rgb)
    assert a.rgb.dtype == np.uint8 and a.rgb.shape == (96, 128, 3) and a.rgb.flags.c_contiguous
    assert a.regions.dtype == np.int32 and a.roi.dtype == bool


def test_noise_table_is_the_discrete_gaussian_of_sigma_6():
    """Thresholds out of 2^32 of P(v) proportional to exp(-v^2 / 72) on -30..30, rounded."""
    v = np.arange(-30, 31)
    p = np.exp(-v.astype(np.float64) ** 2 / 72.0)
    cdf = np.cumsum(p / p.sum())[:-1] * 2.0 ** 32
    np.testing.assert_array_equal(synth._NOISE_CDF.astype(np.int64), np.round(cdf).astype(np.int64))


def test_noise_statistics_on_one_flat_region():
    """One Voronoi cell, no nuclei: the pixels are the region mean plus the noise."""
    img = synth.he_image(256, 256, 1, seed=8, nucleus_density=0.0)  # a purple region: no clipping
    x = img.rgb.astype(np.float64).reshape(-1, 3)
    assert (np.unique(img.regions) == [0]).all()
    m = np.round(x.mean(0))
    assert np.abs(m - synth.PURPLE).max() <= 15
    assert np.abs(x.std(0) - 6.0).max() < 0.1
    assert np.abs(x - m).max() <= 30


def test_class_shares_over_many_regions():
    img = synth.he_image(512, 512, 4000, seed=9, nucleus_density=0.0)
    n = img.n_regions
    mean = np.zeros((n, 3))
    cnt = np.bincount(img.regions.ravel(), minlength=n)
    for c in range(3):
        mean[:, c] = np.bincount(img.regions.ravel(), weights=img.rgb[..., c].ravel(), minlength=n)
    live = cnt > 50
    m = mean[live] / cnt[live, None]
    white = (m > 230).all(1)
    purple = np.abs(m - synth.PURPLE).max(1) < 25
    pink = np.abs(m - synth.PINK).max(1) < 25
    assert (white | purple | pink).all()
    share = np.array([pink.mean(), purple.mean(), white.mean()])
    assert np.abs(share - [0.45, 0.35, 0.20]).max() < 0.04, share
    roi_regions = np.unique(img.regions[img.roi])
    assert set(roi_regions.tolist()) <= set(np.flatnonzero(live)[purple].tolist()) | set(np.flatnonzero(~live).tolist())


def test_nuclei_are_roi_and_avoid_white_regions():
    img = synth.he_image(256, 320, 20, seed=12, white_frac=0.5)
    cells = int(img.regions.max())
    nuc = img.regions >= img.n_regions - int(256 * 320 / 400.0 + 0.5)
    assert nuc.any() and img.roi[nuc].all()
    col = img.rgb[nuc].astype(np.int32).mean(0)
    assert np.abs(col - synth.NUCLEUS).max() < 8
    assert cells < img.n_regions


def test_batch_tile_sizes_follow_the_recipe():
    sizes = synth.batch_sizes(64, 3)
    assert len(sizes) == 64
    for H, W in sizes:
        long_side, short_side = max(H, W), min(H, W)
        assert long_side in (512, 1024, 2048, 3072, 4096)
        assert short_side % 32 == 0 and short_side >= 32
        assert long_side / 2 - 32 < short_side <= long_side
    assert sizes == synth.batch_sizes(64, 3)


def test_slide_folds_cover_the_requested_share():
    img = synth.slide_image(1024, 768, seed=5, fold_frac=0.05)
    base = synth.he_image(1024, 768, max(1, 1024 * 768 // 8192), 5, white_frac=0.40)
    folds = img.regions >= base.n_regions
    assert 0.05 <= folds.mean() < 0.15
    assert not img.roi[folds].any()
    np.testing.assert_array_equal(img.rgb[~folds], base.rgb[~folds])
