"""Exact references for the bit-width 0-1 ILP and the reserve-ratio pick.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Eq. (eq:ilp), Sec. III-F "Binary ILP for Q": one one-hot vector per
(channel i, block j) picks one of Q bit-widths; minimise the quality loss
Omega(Q) subject to the estimated size S(Q) <= budget.  Over a cost table this
is a multiple-choice knapsack.

Size model (Sec. III-F "Size Estimator", Eq. (eq:size_estim)):
    bytes = sum_items rate(item, b) / 8 + 9 * n_items + C_const
with rate = the entropy bound -sum h log2(h/n) of the group (default) or the
fixed-length n * b bits (P_ij * Q_ij); 9 bytes of metadata per group-channel
(FP32 min, FP32 max, one byte of bit-width, Sec. III-G item 4); C_const is the
caller's exact byte count for coordinates and other metadata.

Distortion (Sec. III-F "Acceleration", Omega = |A_hat - A| with the 1-, 2- or
inf-norm): "sse" sums squared errors (default), "l2" sums per-group 2-norms
sqrt(SSE), "l1" and "linf" the other two norms.

Reserve-ratio pick (Alg. 1, read as follows where it is silent): a ratio is
skipped when even the top bit-width everywhere stays under the budget (tau too
small); among the other feasible ratios the smallest total distortion wins,
ties to the larger ratio.  If every feasible ratio is skipped, the largest
feasible ratio is taken.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

META_BYTES_PER_ITEM = 9


def item_rates(table: dict, bits, rate: str = "entropy") -> np.ndarray:
    """[n_items, n_b] rate in bits."""
    if rate == "entropy":
        return np.asarray(table["hbits"], dtype=np.float64)
    if rate == "fixed":
        return np.asarray(table["cnt"], dtype=np.float64)[:, None] * np.asarray(bits, dtype=np.float64)[None, :]
    raise ValueError(rate)


def item_dist(table: dict, norm: str = "sse") -> np.ndarray:
    if norm == "sse":
        return np.asarray(table["sse"], dtype=np.float64)
    if norm == "l2":
        return np.sqrt(np.asarray(table["sse"], dtype=np.float64))
    if norm == "l1":
        return np.asarray(table["l1"], dtype=np.float64)
    if norm == "linf":
        return np.asarray(table["linf"], dtype=np.float64)
    raise ValueError(norm)


def assignment_bytes(rates: np.ndarray, choice: np.ndarray, const_bytes: float) -> float:
    n_items = rates.shape[0]
    return float(rates[np.arange(n_items), choice].sum() / 8.0 + META_BYTES_PER_ITEM * n_items + const_bytes)


def solve_bruteforce(dist: np.ndarray, rates: np.ndarray, budget: float, const_bytes: float = 0.0):
    """Enumerate every assignment (tiny instances only).  Returns (objective, choice) or None."""
    n_items, n_b = dist.shape
    best = None
    for choice in itertools.product(range(n_b), repeat=n_items):
        ch = np.array(choice, dtype=np.int64)
        if assignment_bytes(rates, ch, const_bytes) <= budget:
            obj = float(dist[np.arange(n_items), ch].sum())
            if best is None or obj < best[0]:
                best = (obj, ch)
    return best


def solve_dp_integer(dist: np.ndarray, weights_bits: np.ndarray, budget: float, const_bytes: float = 0.0):
    """Exact DP when every rate is an integer number of bits (fixed-length model).

    Capacity in bits: floor(8 * (budget - 9 * n_items - const)).  Returns (objective, choice) or None.
    """
    n_items, n_b = dist.shape
    w = np.asarray(weights_bits, dtype=np.int64)
    cap_bytes = budget - META_BYTES_PER_ITEM * n_items - const_bytes
    if cap_bytes < 0:
        return None
    cap = int(math.floor(8.0 * cap_bytes))
    INF = np.inf
    dp = np.full(cap + 1, INF)
    dp[0] = 0.0
    back = np.zeros((n_items, cap + 1), dtype=np.int16)
    for i in range(n_items):
        new = np.full(cap + 1, INF)
        arg = np.zeros(cap + 1, dtype=np.int16)
        for k in range(n_b):
            wk = int(w[i, k])
            if wk > cap:
                continue
            cand = np.full(cap + 1, INF)
            cand[wk:] = dp[:cap + 1 - wk] + dist[i, k]
            better = cand < new
            new[better] = cand[better]
            arg[better] = k
        dp = new
        back[i] = arg
    if not np.isfinite(dp).any():
        return None
    end = int(np.argmin(dp))
    obj = float(dp[end])
    choice = np.zeros(n_items, dtype=np.int64)
    c = end
    for i in range(n_items - 1, -1, -1):
        k = int(back[i, c])
        choice[i] = k
        c -= int(w[i, k])
    return obj, choice


def choose_tau(per_r: list[dict], budget: float) -> int | None:
    """Pick the reserve-ratio index from per-ratio results.

    per_r[r] holds: feasible (bool), objective (float), bytes_min, bytes_top (floats).
    """
    feas = [r for r, x in enumerate(per_r) if x["feasible"]]
    if not feas:
        return None
    cands = [r for r in feas if not (per_r[r]["bytes_top"] < budget)]
    if not cands:
        return max(feas)
    best = None
    for r in cands:
        obj = per_r[r]["objective"]
        if best is None or obj < per_r[best]["objective"] or (obj == per_r[best]["objective"] and r > best):
            best = r
    return best
