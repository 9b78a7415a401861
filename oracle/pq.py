"""Oracle product quantisation for OPQ-L, FP64.  TEST INFRASTRUCTURE ONLY.

OPQ-L (Section V-B, "Approximate Distances") takes as approximate distance
the asymmetric distance of OPQ (the query is not quantised; the vector is
its quantised reconstruction) and adds the distance from the vector to its
reconstruction as a third feature of the learned correction.  The paper
uses OPQ with m subspaces and 2^nbit = 256 centroids each (Section VII-A:
m = D/4, D/8 for GIST).

Readings where the paper is silent:
* OPQ's rotation is its parametric solution (Ge, He, Ke and Sun, "Optimized
  Product Quantization", 2014): on the PCA basis, the dimensions are
  allocated to the m subspaces of D/m dimensions each so that the products
  of their variances balance.  The greedy rule (largest variance first, to
  the non-full subspace of smallest product) depends on the scale of the
  variances when subspaces hold different counts, so it is applied round by
  round: the dims, in decreasing variance, are dealt m per round, one to
  each subspace, the larger variances to the subspaces of smaller product so
  far (lower subspace on a tie).  The PCA rotation is the index's, so OPQ's
  rotation is that permutation of it.
* Codebooks: Lloyd k-means in FP64 per subspace from given initial rows,
  a fixed number of iterations, an empty cluster keeps its centroid.
* Encoding: the nearest centroid of each subspace, the lower index on a tie.
* dis' = sum_j ||q_j - c_j,code_j||^2 over the subspaces j (through the
  per-query table lut[j][k] = ||q_j - c_jk||^2); e = ||x - reconstruction||,
  x the stored vector.
"""
from __future__ import annotations

import math

import numpy as np

from . import ivf

KSUB = 256


def eigen_allocation(var: np.ndarray, m: int) -> np.ndarray:
    """Dims of subspace j are perm[j*ds:(j+1)*ds] (ascending), ds = D/m."""
    var = np.asarray(var, dtype=np.float64)
    D = len(var)
    assert D % m == 0
    ds = D // m
    order = np.argsort(-var, kind="stable")
    logp = np.zeros(m)
    groups = [[] for _ in range(m)]
    for t in range(ds):
        dims = order[t * m:(t + 1) * m]                  # decreasing variance
        subs = sorted(range(m), key=lambda j: (logp[j], j))  # increasing product
        for d, j in zip(dims, subs):
            groups[j].append(int(d))
            logp[j] += math.log(max(float(var[d]), 1e-300))
    return np.concatenate([np.sort(np.asarray(g, dtype=np.int64)) for g in groups])


def train_codebooks(Xs: np.ndarray, perm: np.ndarray, m: int, iters: int, init_rows: np.ndarray) -> np.ndarray:
    """codebooks[m, 256, ds] by k-means on the subspaces of Xs (n x D)."""
    Xs = np.asarray(Xs, dtype=np.float64)
    ds = Xs.shape[1] // m
    cb = np.empty((m, KSUB, ds))
    for j in range(m):
        sub = Xs[:, perm[j * ds:(j + 1) * ds]]
        C, _, _ = ivf.kmeans(sub, np.asarray(init_rows), iters)
        cb[j] = C
    return cb


def encode(Xs: np.ndarray, perm: np.ndarray, cb: np.ndarray) -> np.ndarray:
    """codes[n, m] (uint8): nearest centroid per subspace, lower index on a tie."""
    Xs = np.asarray(Xs, dtype=np.float64)
    m, _, ds = cb.shape
    codes = np.empty((Xs.shape[0], m), dtype=np.uint8)
    for j in range(m):
        sub = Xs[:, perm[j * ds:(j + 1) * ds]]
        codes[:, j] = ivf.assign(sub, cb[j])
    return codes


def reconstruct(codes: np.ndarray, perm: np.ndarray, cb: np.ndarray) -> np.ndarray:
    m, _, ds = cb.shape
    out = np.zeros((codes.shape[0], m * ds))
    for j in range(m):
        out[:, perm[j * ds:(j + 1) * ds]] = cb[j][codes[:, j]]
    return out


def quantisation_error(Xs: np.ndarray, codes: np.ndarray, perm: np.ndarray, cb: np.ndarray) -> np.ndarray:
    """e = ||x - reconstruction|| per row."""
    diff = np.asarray(Xs, dtype=np.float64) - reconstruct(codes, perm, cb)
    return np.sqrt(np.einsum("ij,ij->i", diff, diff))


def lut(Qr: np.ndarray, perm: np.ndarray, cb: np.ndarray) -> np.ndarray:
    """lut[b, j, k] = ||q_j - c_jk||^2 for every query row."""
    Qr = np.asarray(Qr, dtype=np.float64)
    m, K, ds = cb.shape
    out = np.empty((Qr.shape[0], m, K))
    for j in range(m):
        sub = Qr[:, perm[j * ds:(j + 1) * ds]]
        out[:, j, :] = ((sub[:, None, :] - cb[j][None, :, :]) ** 2).sum(-1)
    return out


def asymmetric_distance(table: np.ndarray, codes: np.ndarray) -> np.ndarray:
    """dis'[n] = sum_j table[j, codes[:, j]] for one query's table[m, 256]."""
    m = table.shape[0]
    return table[np.arange(m)[None, :], codes.astype(np.int64)].sum(1)
