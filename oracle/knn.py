"""Nearest-neighbour distance of every point, the scale initialisation of Sec. 3.2
(TEST INFRASTRUCTURE ONLY).

Sec. 3.2 initialises every point's scale isotropically with s_i = min over the other points
p of |p_i - p|_2.  ``nn_distance_brute`` states that definition directly in FP64 (all
pairs, in chunks); ``nn_distance_tree`` answers the same query with scipy's k-d tree (a
library routine, exact for the 2 nearest neighbours: the first is the point itself or a
duplicate at distance 0), for sizes where all pairs are too many.  ``init_log_scales``
turns the distances into the log-scale parameters (3 equal rows), with distances floored
at 1e-7 so that duplicated points get a finite scale.
Pins: tests/test_oracle_knn.py.
"""
from __future__ import annotations

import numpy as np

DIST_FLOOR = 1e-7


def nn_distance_brute(points: np.ndarray, chunk: int = 512) -> np.ndarray:
    """points [n, 3] -> min_{j != i} |p_i - p_j| in FP64."""
    p = np.asarray(points, np.float64)
    n = p.shape[0]
    out = np.empty(n)
    for s in range(0, n, chunk):
        d2 = ((p[s:s + chunk, None, :] - p[None, :, :]) ** 2).sum(-1)
        d2[np.arange(min(chunk, n - s)), np.arange(s, min(s + chunk, n))] = np.inf
        out[s:s + chunk] = np.sqrt(d2.min(1))
    return out


def nn_distance_tree(points: np.ndarray) -> np.ndarray:
    from scipy.spatial import cKDTree
    p = np.asarray(points, np.float64)
    d, _ = cKDTree(p).query(p, k=2)
    return d[:, 1]


def init_log_scales(nn_dist: np.ndarray) -> np.ndarray:
    """[3, n] log-scales of isotropic Gaussians with s_i = max(nn distance, 1e-7)."""
    s = np.maximum(np.asarray(nn_dist, np.float64), DIST_FLOOR)
    return np.repeat(np.log(s)[None], 3, axis=0)
