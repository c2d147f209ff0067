"""Segmentation quality measures that judge a refinement against ground truth or against
the plain method (evaluation only; nothing here takes part in the refinement):

* boundary recall: the fraction of ground-truth boundary pixels with a superpixel
  boundary pixel within ``tol`` pixels (Euclidean);
* undersegmentation error: for every (superpixel, ground-truth region) pair the smaller
  of the overlap and the rest of the superpixel, summed over pairs, over the image size;
* disagreement: the fraction of pixels whose label differs between two label maps of the
  same seeding (label ids are stable, so equal ids mean the same superpixel).

A pixel is a boundary pixel when its right or lower 4-neighbour has another label.
"""
from __future__ import annotations

import numpy as np
import scipy.ndimage as ndi


def boundary_map(lab: np.ndarray) -> np.ndarray:
    b = np.zeros(lab.shape, bool)
    b[:, :-1] |= lab[:, :-1] != lab[:, 1:]
    b[:-1, :] |= lab[:-1, :] != lab[1:, :]
    return b


def boundary_recall(lab: np.ndarray, gt: np.ndarray, tol: int = 2) -> float:
    gb = boundary_map(gt)
    if not gb.any():
        return 1.0
    d = ndi.distance_transform_edt(~boundary_map(lab))
    return float((d[gb] <= tol).mean())


def undersegmentation_error(lab: np.ndarray, gt: np.ndarray) -> float:
    g = int(gt.max()) + 1
    pairs = lab.astype(np.int64).ravel() * g + gt.ravel()
    u, c = np.unique(pairs, return_counts=True)
    sp = u // g
    spsz = np.bincount(lab.ravel().astype(np.int64))
    return float(np.minimum(c, spsz[sp] - c).sum() / lab.size)


def disagreement(a: np.ndarray, b: np.ndarray) -> float:
    return float((a != b).mean())
