"""Shared helpers of the parity tests: seeded setups, comparisons, oracle runs."""
from __future__ import annotations

import numpy as np

from oracle import operator as O


def normwise_rel(a, b) -> float:
    """max |a - b| / max |b| (b is the reference)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def decide_f32(z, theta_pos, theta_neg, kind="filter", bias=None):
    """The label head's decision taken in float32 like the kernel (ties: unsure, then reject)."""
    z = np.asarray(z, dtype=np.float32)
    if kind == "classify":
        b = np.zeros(z.shape[1], np.float32) if bias is None else np.asarray(bias, np.float32)
        v = z + b
        return np.argmax(v, axis=1).astype(np.int32)
    s = (z[:, 0] - z[:, 1]).astype(np.float32)
    a = (s - np.float32(theta_pos)).astype(np.float32)
    rj = (np.float32(theta_neg) - s).astype(np.float32)
    u = np.float32(0)
    out = np.where((u >= a) & (u >= rj), O.UNSURE, np.where(rj >= a, O.REJECT, O.ACCEPT))
    return out.astype(np.int32)


def check_retained_vs_oracle(gpu_idx, oracle_scores, n):
    """Retained sets against the oracle's ranking: equal except at near-ties of the
    oracle scores at the rank boundary (FP32 vs FP64 scoring).  Returns the number of
    exchanged pairs."""
    s = np.asarray(oracle_scores, dtype=np.float64)
    ref = O.rank_order(s)[:n]
    a, b = set(int(x) for x in gpu_idx[:n]), set(int(x) for x in ref)
    diff = a ^ b
    if not diff:
        return 0
    kth = s[ref[-1]]
    tol = 1e-5 * max(1.0, abs(kth))   # boundary near-tie band
    for j in diff:
        assert abs(s[j] - kth) <= tol, (j, s[j], kth)
    return len(diff) // 2
