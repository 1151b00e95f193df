"""FP64 statement of the optimisation step around the hot path (TEST INFRASTRUCTURE ONLY).

Sec. 3.2 optimises the point parameters phi as 3D Gaussian Splatting does, with Adam
(Kingma & Ba, "Adam: A Method for Stochastic Optimization", Algorithm 1), and Sec. 3.3
removes the points whose importance is below t_prune twice during optimisation.  This
module states both plainly in numpy FP64:

* ``adam`` -- one step of Algorithm 1 on a parameter array: with g the gradient and t the
  step number (1-based), m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
  m_hat = m / (1 - b1^t), v_hat = v / (1 - b2^t), p <- p - lr m_hat / (sqrt(v_hat) + eps);
* ``prune`` -- the survivors of the pruning mask m_i = 1(h_i < t): the indices with
  h_i >= t in ascending order, and every parameter array (and optimiser moment) reduced to
  those columns, in that order.

Pins: tests/test_oracle_optim.py.
"""
from __future__ import annotations

from typing import Dict, Sequence, Tuple

import numpy as np


def adam(p, g, m, v, lr: float, step: int, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-15):
    """One Adam step (Algorithm 1 of Kingma & Ba) in FP64.  Returns new (p, m, v)."""
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def survivors(h, t: float) -> np.ndarray:
    """Ascending indices i with h_i >= t (the complement of the pruning mask 1(h < t))."""
    h = np.asarray(h)
    return np.nonzero(~(h < np.float32(t)))[0].astype(np.uint32)


def prune(arrays: Dict[str, np.ndarray], h, t: float) -> Tuple[np.ndarray, Dict[str, np.ndarray]]:
    """Every array (rows x N, SoA) reduced to the survivors' columns, in ascending order."""
    keep = survivors(h, t)
    return keep, {k: np.asarray(a)[..., keep.astype(np.int64)] for k, a in arrays.items()}
