"""Lloyd's k-means on camera positions, as the clustering step of Sec. 3.4 uses it
(TEST INFRASTRUCTURE ONLY).

Sec. 3.4 runs k-means on the input camera locations and assigns every camera to its
cluster centre.  Stated plainly (Lloyd's algorithm, fixed iteration count, caller-given
initial centres):
  repeat `iterations` times:
    assign every point to the nearest centre: the FP32 squared distance
      ((x0 - c0)^2 + (x1 - c1)^2) + (x2 - c2)^2 (each operation rounded to FP32), ties to the
      lower centre index;
    move every centre with at least one point to the mean of its points (the sum in FP64,
      divided by the count in FP64, rounded to FP32); a centre without points stays.
  finally assign once more with the final centres.
Pins: tests/test_oracle_kmeans.py.
"""
from __future__ import annotations

import numpy as np


def assign(points: np.ndarray, centres: np.ndarray) -> np.ndarray:
    p = np.asarray(points, np.float32)
    c = np.asarray(centres, np.float32)
    d0 = (p[:, None, 0] - c[None, :, 0]).astype(np.float32)
    d1 = (p[:, None, 1] - c[None, :, 1]).astype(np.float32)
    d2 = (p[:, None, 2] - c[None, :, 2]).astype(np.float32)
    d = (d0 * d0).astype(np.float32)
    d = (d + (d1 * d1).astype(np.float32)).astype(np.float32)
    d = (d + (d2 * d2).astype(np.float32)).astype(np.float32)
    return np.argmin(d, axis=1).astype(np.int32)   # argmin takes the first (lowest) index on ties


def kmeans(points: np.ndarray, init: np.ndarray, iterations: int):
    """Returns (centres [k, 3] float32, assignment [n] int32)."""
    p = np.asarray(points, np.float32)
    c = np.asarray(init, np.float32).copy()
    for _ in range(iterations):
        a = assign(p, c)
        for j in range(c.shape[0]):
            members = p[a == j].astype(np.float64)
            if len(members):
                c[j] = (members.sum(axis=0) / len(members)).astype(np.float32)
    return c, assign(p, c)
