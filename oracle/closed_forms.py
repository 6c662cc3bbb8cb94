"""FP64 oracle, part 3: closed-form optima used to pin the iterative solvers.

TEST INFRASTRUCTURE ONLY (see ``oracle.model``).

With one cell and one user (C = K = 1) problem (1) is the point-to-point MIMO
capacity under a sum-power budget, whose optimum is the eigen-beamforming
water-filling solution over the singular values of H.  When users see the BS
through disjoint antenna subsets (no interference), problem (1) with alpha = 1
separates into the same water-filling over the union of every user's
singular values.  Neither uses any step of the iterative algorithms.
"""
from __future__ import annotations

import numpy as np


def waterfill(gains: np.ndarray, P: float, sigma2: float) -> np.ndarray:
    """Powers p_m = (mu - sigma2/g_m)^+ with sum p = P for channel gains g_m."""
    g = np.sort(np.asarray(gains, dtype=np.float64))[::-1]
    g = g[g > 0]
    inv = sigma2 / g
    for n in range(len(g), 0, -1):
        mu = (P + np.sum(inv[:n])) / n
        if mu > inv[n - 1]:
            p = np.zeros(len(g))
            p[:n] = mu - inv[:n]
            return p
    return np.zeros(len(g))


def capacity_nats(gains: np.ndarray, P: float, sigma2: float) -> float:
    """sum_m log(1 + p_m g_m / sigma2) at the water-filling powers."""
    g = np.sort(np.asarray(gains, dtype=np.float64))[::-1]
    g = g[g > 0]
    p = waterfill(g, P, sigma2)
    return float(np.sum(np.log1p(p * g / sigma2)))


def single_user_capacity(H: np.ndarray, P: float, sigma2: float, d: int) -> float:
    """Capacity with at most d streams: water-filling over the d largest
    squared singular values of H (Nr x Nt)."""
    s = np.linalg.svd(H, compute_uv=False)
    return capacity_nats(s[:d] ** 2, P, sigma2)


def miso_mrt_rate(h: np.ndarray, P: float, sigma2: float) -> float:
    """Single-antenna user, one stream: log(1 + P ||h||^2 / sigma2)."""
    return float(np.log1p(P * np.sum(np.abs(h) ** 2) / sigma2))
