"""The segmentation quality measures (boundary recall, undersegmentation error,
disagreement) against closed forms on hand-made label maps."""
import numpy as np
import pytest

from paper_1704_02083_gb300.quality import boundary_map, boundary_recall, disagreement, undersegmentation_error


def _split(H, W, x0):
    return np.where(np.arange(W)[None, :] < x0, 0, 1) * np.ones((H, 1), np.int64)


def test_boundary_map_marks_the_left_and_upper_side():
    lab = _split(4, 6, 3)
    b = boundary_map(lab)
    assert b[:, 2].all() and b.sum() == 4


def test_recall_of_ground_truth_against_itself_is_one():
    gt = np.add.outer(np.arange(20) // 5, 4 * (np.arange(30) // 7))
    assert boundary_recall(gt, gt) == 1.0


@pytest.mark.parametrize("shift,tol,want", [(0, 0, 1.0), (2, 2, 1.0), (3, 2, 0.0), (2, 1, 0.0), (1, 1, 1.0)])
def test_recall_tolerance_is_a_euclidean_distance(shift, tol, want):
    """A vertical edge found `shift` columns away counts when shift <= tol."""
    gt = _split(16, 32, 12)
    lab = _split(16, 32, 12 + shift)
    assert boundary_recall(lab, gt, tol) == want


def test_recall_counts_the_fraction_of_boundary_found():
    """Ground truth with two vertical edges; the segmentation finds one of them."""
    gt = np.where(np.arange(40)[None, :] < 10, 0, np.where(np.arange(40)[None, :] < 30, 1, 2)) * np.ones((8, 1), int)
    lab = _split(8, 40, 10)
    assert boundary_recall(lab, gt, 0) == 0.5


def test_recall_without_ground_truth_boundary_is_one():
    assert boundary_recall(_split(8, 8, 4), np.zeros((8, 8), int)) == 1.0


def test_undersegmentation_closed_forms():
    H, W = 10, 20
    gt = _split(H, W, 6)  # regions of 60 and 140 pixels
    assert undersegmentation_error(gt, gt) == 0.0
    one = np.zeros((H, W), int)
    # one superpixel over both regions: min(60, 140) + min(140, 60) over 200 pixels
    assert undersegmentation_error(one, gt) == pytest.approx(120 / 200)
    # a superpixel that leaks 2 columns (20 pixels) into the larger region
    lab = _split(H, W, 8)
    assert undersegmentation_error(lab, gt) == pytest.approx((20 + 20) / 200)
    # ids are names: a permutation of the superpixel ids changes nothing
    perm = np.array([7, 3])
    assert undersegmentation_error(perm[lab], gt) == undersegmentation_error(lab, gt)


def test_disagreement_is_the_fraction_of_pixels_that_differ():
    a = _split(10, 10, 5)
    b = _split(10, 10, 7)
    assert disagreement(a, a) == 0.0
    assert disagreement(a, b) == pytest.approx(20 / 100)
