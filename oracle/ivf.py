"""Oracle IVF candidate generation, FP64 (Section II-A).

IVF clusters the database with k-means into nlist buckets; a query probes the
buckets of its nprobe nearest centroids, and the union of their members is
its candidate set.

Readings (the paper prints no recipe): Lloyd iterations from a given set of
initial rows; a point goes to the centroid of smallest squared distance, the
lower centroid id on a tie; an empty cluster keeps its previous centroid;
probes are ordered by (distance, list id).  Distances are computed directly
as sum((a - b)^2), not by the norm expansion.
"""
from __future__ import annotations

import numpy as np


def sq_dists(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """All-pairs squared L2 distances sum_j (a_j - b_j)^2, FP64, direct form."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    out = np.empty((A.shape[0], B.shape[0]))
    step = max(1, (1 << 22) // max(1, B.shape[0] * A.shape[1]))
    for a in range(0, A.shape[0], step):
        d = A[a:a + step, None, :] - B[None, :, :]
        out[a:a + step] = np.einsum("ijk,ijk->ij", d, d)
    return out


def assign(Xr: np.ndarray, C: np.ndarray) -> np.ndarray:
    """argmin_j ||x - c_j||^2 per row; np.argmin returns the lowest index on ties."""
    return np.argmin(sq_dists(Xr, C), axis=1).astype(np.int32)


def kmeans(Xr: np.ndarray, init_rows: np.ndarray, iters: int):
    """Lloyd's algorithm in FP64.  Returns (centroids, assignment, objectives)
    where objectives[t] is the mean squared distance to the assigned centroid
    after the t-th assignment step."""
    Xd = np.asarray(Xr, dtype=np.float64)
    C = Xd[np.asarray(init_rows)].copy()
    objs = []
    a = None
    for _ in range(iters):
        d = sq_dists(Xd, C)
        a = np.argmin(d, axis=1)
        objs.append(float(d[np.arange(len(a)), a].mean()))
        for j in range(C.shape[0]):
            m = a == j
            if m.any():
                C[j] = Xd[m].mean(axis=0)
    d = sq_dists(Xd, C)
    a = np.argmin(d, axis=1)
    objs.append(float(d[np.arange(len(a)), a].mean()))
    return C, a.astype(np.int32), objs


def probe(Qr: np.ndarray, C: np.ndarray, nprobe: int):
    """The nprobe nearest centroids per query, ordered by (distance, list id).
    Returns (lists[B, nprobe] int32, dists[B, nprobe] FP64)."""
    d = sq_dists(Qr, C)
    ids = np.arange(C.shape[0])
    out = np.empty((d.shape[0], nprobe), dtype=np.int32)
    od = np.empty((d.shape[0], nprobe))
    for b in range(d.shape[0]):
        o = np.lexsort((ids, d[b]))[:nprobe]
        out[b] = o
        od[b] = d[b, o]
    return out, od


def lists_from_assignment(assign_: np.ndarray, nlist: int):
    """Bucket members in storage order: lists in id order, members of a list
    in increasing row order.  Returns (offsets[nlist+1], members[N])."""
    a = np.asarray(assign_, dtype=np.int64)
    members = np.argsort(a, kind="stable").astype(np.int64)
    counts = np.bincount(a, minlength=nlist)
    offsets = np.zeros(nlist + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    return offsets, members
