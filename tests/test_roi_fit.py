"""Host side of the linear classifier of Eq. predict (roi.py): the balanced sampling of
Sec. 4.1 and the logistic fit, on synthetic feature sets whose separating rule is known."""
import numpy as np

from paper_1704_02083_gb300 import roi


def _data(n, theta, seed, noise=0.0):
    rng = np.random.default_rng(seed)
    F = np.column_stack([rng.uniform(0, 255, n), rng.normal(0, 30, n), rng.uniform(0, 100, n), rng.uniform(0, 60, n)])
    h = theta[0] + F @ theta[1:] + rng.normal(0, noise, n)
    return F, np.where(h >= 0, 1, -1).astype(np.int8)


def _predict(theta, F):
    h = (((theta[0] + theta[1] * F[:, 0]) + theta[2] * F[:, 1]) + theta[3] * F[:, 2]) + theta[4] * F[:, 3]
    return np.where(h >= 0, 1, -1)


def test_fit_recovers_a_linear_rule_in_feature_units():
    true = np.array([300.0, -2.0, 0.5, 1.5, -1.0])
    F, y = _data(4000, true, 1)
    theta, info = roi.fit(F, y, seed=0)
    assert info["samples"] == 2 * min((y > 0).sum(), (y < 0).sum())  # half positive, half negative
    assert (_predict(theta, F) == y).mean() > 0.99
    # the same direction as the true rule (up to scale)
    cos = theta @ true / np.linalg.norm(theta) / np.linalg.norm(true)
    assert cos > 0.95


def test_balanced_sampling_keeps_a_rare_class():
    true = np.array([-200.0, 1.0, 0.0, 0.0, 0.0])  # ROI only above brightness 200: ~22% of samples
    F, y = _data(3000, true, 2, noise=5.0)
    theta, info = roi.fit(F, y, seed=3)
    assert info["positives"] < info["negatives"]
    assert roi.balanced_accuracy(_predict(theta, F), y) > 0.9


def test_ground_truth_is_the_majority_class():
    lab = np.array([[0, 0, 1, 1], [0, 2, 1, 1]], np.int32)
    roi_mask = np.array([[1, 0, 1, 1], [1, 1, 0, 0]], bool)
    y, n = roi.ground_truth(lab, roi_mask, 4)
    # label 0: 2 of 3 ROI; label 1: 2 of 4 (half counts as ROI); label 2: 1 of 1; label 3: empty
    assert y.tolist()[:3] == [1, 1, 1] and n.tolist() == [3, 4, 1, 0]
    y2, _ = roi.ground_truth(lab, ~roi_mask, 4)
    assert y2.tolist()[:3] == [-1, 1, -1]
