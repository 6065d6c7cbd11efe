"""Split a batch of independent NMPC instances over the GPUs of one node.

The instances of a batch are independent problems (their KKT systems are the
diagonal blocks of one block-diagonal system), so the batch shards with no
exchange: each rank builds and solves a contiguous range of instances.  The
ranges are balanced by the work of one numeric factorization of each
instance, the floating-point operations the one-time structure analysis
reports for its horizon (the factorization dominates an interior-point
iteration), so that the slowest rank, which sets the job's time, carries as
little extra as the contiguity allows.
"""
from __future__ import annotations

import numpy as np


def instance_weights(model, horizons, opts=None, **prob_kw):
    """Factorization flops of each instance, from the host-only structure
    analysis of one instance per distinct horizon (no device memory)."""
    from ._lib import Structure
    hz = np.asarray(horizons, dtype=np.int64)
    cache = {}
    for T in np.unique(hz):
        s = Structure(model, [int(T)], opts=opts, **prob_kw)
        cache[int(T)] = float(s.stats()["factor_flops"])
        s.close()
    return np.array([cache[int(T)] for T in hz])


def contiguous_partition(weights, parts):
    """Cut 0..len(weights) into `parts` contiguous ranges [b_r, b_{r+1}) whose
    weight sums are as even as the contiguous order allows: cut r goes where
    the running sum is closest to r/parts of the total, never leaving a range
    empty while instances remain.  Returns the parts + 1 boundaries."""
    w = np.asarray(weights, dtype=np.float64)
    n = w.size
    if parts < 1:
        raise ValueError("parts must be >= 1")
    if n < parts:
        raise ValueError("fewer instances than ranks")
    if np.any(w < 0):
        raise ValueError("weights must be non-negative")
    c = np.concatenate([[0.0], np.cumsum(w)])
    total = c[-1]
    b = [0]
    for r in range(1, parts):
        target = total * r / parts
        k = int(np.searchsorted(c, target))
        if k > 0 and abs(c[k - 1] - target) <= abs(c[min(k, n)] - target):
            k -= 1
        lo, hi = b[-1] + 1, n - (parts - r)  # every range keeps at least one instance
        b.append(int(min(max(k, lo), hi)))
    b.append(n)
    return b


def rank_slice(weights, rank, world):
    """(first, end) instance range of `rank` among `world` ranks."""
    b = contiguous_partition(weights, world)
    return b[rank], b[rank + 1]
