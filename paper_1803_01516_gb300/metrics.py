"""Accuracy report of §4.2 (Eq. 2) against a synthetic ground truth.

Not on the solver path: it reads the labels the solver returns and the
ground-truth disparity map the scene generator draws.
"""
from __future__ import annotations

import numpy as np


def gt_depth(dR: np.ndarray, D: int, dis0: int) -> np.ndarray:
    """Ground-truth depth number of every site (W, y).

    Along gaze line W the cross point of depth number S pairs right pixel
    x_r = W + S with disparity dis(S) = dis0 - 2S (§4.1).  The true depth is
    the first cross point, from the front, that is at or behind the visible
    surface: the smallest S with dis(S) <= d_R(W + S, y), else D - 1.  Only
    every other disparity is representable (§4.1), so an odd disparity d maps
    to dis = d - 1, i.e. the division by 2 rounds away from the front.
    """
    dR = np.asarray(dR)
    h, w = dR.shape
    ng = w - dis0
    gt = np.full((h, ng), D - 1, dtype=np.int32)
    for S in range(D - 1, -1, -1):
        ok = (dis0 - 2 * S) <= dR[:, S:S + ng]
        gt = np.where(ok, S, gt)
    return gt


def depth_error_hist(labels: np.ndarray, gt: np.ndarray) -> np.ndarray:
    """Number of sites at each depth-number difference d(s) = |X_s - gt_s|."""
    d = np.abs(np.asarray(labels, dtype=np.int64) - np.asarray(gt, dtype=np.int64))
    return np.bincount(d.ravel())


def depth_error_from_hist(hist) -> int:
    """Eq. 2: error = sum_d d x (number of sites with difference d)."""
    hist = np.asarray(hist, dtype=np.int64)
    return int((np.arange(hist.size) * hist).sum())


def depth_error(labels: np.ndarray, gt: np.ndarray):
    """(error of Eq. 2, fraction of sites equal to the ground truth)."""
    hist = depth_error_hist(labels, gt)
    return depth_error_from_hist(hist), float(hist[0]) / max(int(hist.sum()), 1)
