"""Oracle exact KNN by brute force, FP64 (Section II-A).

dis(p, q) = ||p - q||^2; the K nearest are the K smallest, ordered by
(distance, id) so that ties are resolved by the lower id.
"""
from __future__ import annotations

import numpy as np


def exact_knn(X: np.ndarray, Q: np.ndarray, K: int, ids: np.ndarray | None = None):
    """Returns (ids[B, K] int64, dists[B, K] FP64) of the K nearest rows of X."""
    X = np.asarray(X, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    ids = np.arange(X.shape[0], dtype=np.int64) if ids is None else np.asarray(ids, np.int64)
    K = min(K, X.shape[0])
    out_i = np.empty((Q.shape[0], K), dtype=np.int64)
    out_d = np.empty((Q.shape[0], K))
    step = max(1, (1 << 23) // max(1, X.shape[0]))
    for a in range(0, Q.shape[0], step):
        q = Q[a:a + step]
        # direct form, summed per row: exact up to FP64 rounding of the sum
        for b in range(q.shape[0]):
            diff = X - q[b][None, :]
            d = np.einsum("ij,ij->i", diff, diff)
            o = np.lexsort((ids, d))[:K]
            out_i[a + b] = ids[o]
            out_d[a + b] = d[o]
    return out_i, out_d
