"""Independent checks used by the tests (no code shared with the oracle or the CUDA path)."""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import scipy.ndimage as ndi
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components


def stats_from_labels(rgb: np.ndarray, lab_full: np.ndarray, M: int) -> np.ndarray:
    """Per-label (N, sumR, sumG, sumB, sumX, sumY) from a full-res label map, in int64."""
    H, W = lab_full.shape
    L = lab_full.ravel().astype(np.int64)
    yy, xx = np.mgrid[0:H, 0:W]
    out = np.zeros((M, 6), np.int64)
    out[:, 0] = np.bincount(L, minlength=M)
    for c in range(3):
        out[:, 1 + c] = np.bincount(L, weights=rgb[..., c].ravel().astype(np.float64), minlength=M).astype(np.int64)
    # positions can exceed 2^53 only for huge images; the tests stay far below
    out[:, 4] = np.bincount(L, weights=xx.ravel().astype(np.float64), minlength=M).astype(np.int64)
    out[:, 5] = np.bincount(L, weights=yy.ravel().astype(np.float64), minlength=M).astype(np.int64)
    return out


def upsample(block_lab: np.ndarray, side: int, H: int, W: int) -> np.ndarray:
    return np.repeat(np.repeat(block_lab, side, 0), side, 1)[:H, :W]


def count_components_per_label(lab: np.ndarray) -> int:
    """Number of 4-connected components of equal-label regions (all labels together)."""
    H, W = lab.shape
    idx = np.arange(H * W).reshape(H, W)
    rows, cols = [], []
    m = lab[:, :-1] == lab[:, 1:]
    rows.append(idx[:, :-1][m]); cols.append(idx[:, 1:][m])
    m = lab[:-1, :] == lab[1:, :]
    rows.append(idx[:-1, :][m]); cols.append(idx[1:, :][m])
    r = np.concatenate(rows); c = np.concatenate(cols)
    g = coo_matrix((np.ones(r.size, np.int8), (r, c)), shape=(H * W, H * W))
    n, _ = connected_components(g, directed=False)
    return n


def unequal_pairs(lab: np.ndarray) -> int:
    return int((lab[:, :-1] != lab[:, 1:]).sum() + (lab[:-1, :] != lab[1:, :]).sum())


def total_energy(rgb: np.ndarray, lab: np.ndarray, lam_pos: float, lam_b: float) -> Fraction:
    """Eq. equa:energy1 at the centroid means, exactly (rational arithmetic):
    sum_k [Q_k - |S_k|^2 / N_k] + lam_pos sum_k [Qp_k - |P_k|^2 / N_k] + 2 lam_b #unequal pairs."""
    H, W = lab.shape
    L = lab.ravel().astype(np.int64)
    yy, xx = np.mgrid[0:H, 0:W]
    E_col = Fraction(0)
    E_pos = Fraction(0)
    labels = np.unique(L)
    order = np.argsort(L, kind="stable")
    Ls = L[order]
    bounds = np.searchsorted(Ls, labels), np.searchsorted(Ls, labels, side="right")
    px = rgb.reshape(-1, 3).astype(np.int64)[order]
    pos = np.stack([xx.ravel(), yy.ravel()], 1).astype(np.int64)[order]
    for a, b in zip(*bounds):
        n = int(b - a)
        S = px[a:b].sum(0)
        Q = int((px[a:b] ** 2).sum())
        E_col += Fraction(Q * n - int((S.astype(object) ** 2).sum()), n)
        P = pos[a:b].sum(0)
        Qp = int((pos[a:b] ** 2).sum())
        E_pos += Fraction(Qp * n - int((P.astype(object) ** 2).sum()), n)
    return E_col + Fraction(lam_pos) * E_pos + 2 * Fraction(lam_b) * unequal_pairs(lab)


# the quality measures live with the package's evaluation code
from paper_1704_02083_gb300.quality import boundary_map, boundary_recall, undersegmentation_error  # noqa: E402,F401
