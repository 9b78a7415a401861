"""Comparison rules between the CUDA path and the oracle.

* Distances: a returned FP32 distance must be within
  1e-5 * max(dis, 1e-3 * median) of the FP64 exact distance of the same id.
* Ids: for a query whose oracle run had no ambiguous test (a learned test
  whose left side fell within delta * tau of tau, which another rounding
  could flip), the ids must equal the oracle's at every rank whose oracle
  distance is separated from its neighbours by more than 1e-5 relative.
* Every query: ids unique, distances non-decreasing, padding -1 / +inf
  exactly where the oracle pads.
"""
import numpy as np

REL = 1e-5


def exact_fp64(X, Q, ids):
    d = np.full(ids.shape, np.inf)
    for b in range(ids.shape[0]):
        v = ids[b] >= 0
        if v.any():
            diff = X[ids[b][v]].astype(np.float64) - Q[b].astype(np.float64)[None, :]
            d[b][v] = np.einsum("ij,ij->i", diff, diff)
    return d


def check(gpu_ids, gpu_d, ora_ids, ora_d, X, Q, K, amb=None, id_of_row=None, min_strict=0.9):
    """Returns (n_strict, n_queries); raises AssertionError on a violation."""
    B = gpu_ids.shape[0]
    K = np.broadcast_to(np.asarray(K), (B,))
    rows_of = (lambda i: i) if id_of_row is None else id_of_row
    ex = exact_fp64(X, Q, np.where(gpu_ids >= 0, rows_of(np.maximum(gpu_ids, 0)), -1))
    strict = 0
    for b in range(B):
        k = int(K[b])
        gi, gd = gpu_ids[b, :k], gpu_d[b, :k]
        oi, od = ora_ids[b, :k], ora_d[b, :k]
        gv, ov = gi >= 0, oi >= 0
        assert len(set(gi[gv].tolist())) == gv.sum(), f"query {b}: duplicate ids"
        assert np.all(np.diff(gd[gv]) >= 0), f"query {b}: distances not sorted"
        assert np.all(np.isinf(gd[~gv])), f"query {b}: padding distance"
        med = np.median(od[ov]) if ov.any() else 1.0
        tol = REL * np.maximum(ex[b, :k][gv], 1e-3 * med)
        err = np.abs(gd[gv].astype(np.float64) - ex[b, :k][gv])
        assert np.all(err <= tol), f"query {b}: distance error {err.max()} > {tol[np.argmax(err - tol)]}"
        if amb is not None and amb[b] > 0:
            continue
        strict += 1
        assert gv.sum() == ov.sum(), f"query {b}: {gv.sum()} results vs oracle {ov.sum()}"
        for r in range(int(ov.sum())):
            lo = r == 0 or od[r] - od[r - 1] > REL * od[r]
            hi = r == ov.sum() - 1 or od[r + 1] - od[r] > REL * od[r + 1]
            if lo and hi:
                assert gi[r] == oi[r], f"query {b} rank {r}: id {gi[r]} vs oracle {oi[r]}"
    assert strict >= min_strict * B, f"only {strict} of {B} queries unambiguous"
    return strict, B


def recall(ids, gt, k):
    return float(np.mean([len(set(ids[b, :k].tolist()) & set(gt[b, :k].tolist())) / k
                          for b in range(len(ids))]))
