"""Comparison rules between the CUDA path and the oracle.

* Distances: every returned FP32 distance must be within
  1e-5 * max(dis, 1e-3 * median) of the FP64 exact distance of the same id
  (with exact_ties: equal to the oracle's, bit for bit, on the ranks below).
* Ids, rank by rank: the oracle reports per query amb_d, the smallest exact
  distance of a candidate whose decision another rounding could flip
  (directly, or through the tau of later waves).  Below amb_d both sides
  hold the same entries, so at every oracle rank whose distance is below
  amb_d the ids must be equal -- where the oracle's distances are separated
  from their neighbours by more than 1e-5 relative (FP32 may order closer
  ones differently), or at every such rank when exact_ties (integer data:
  distances are exact in FP32 on both sides and ties go to the lower id).
  No query is exempt: a query with an uncertain candidate is still checked
  up to that candidate's distance.
* Every query: ids unique, distances non-decreasing, padding -1 / +inf.
* The number of ranks checked is returned; the caller asserts its share.
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


def check(gpu_ids, gpu_d, ora_ids, ora_d, X, Q, K, amb_d=None, id_of_row=None, exact_ties=False,
          min_checked=0.95):
    """Returns (ranks checked, oracle ranks); raises AssertionError on a
    violation or when fewer than min_checked of the oracle's ranks could be
    checked."""
    B = gpu_ids.shape[0]
    K = np.broadcast_to(np.asarray(K), (B,))
    amb_d = np.full(B, np.inf) if amb_d is None else np.asarray(amb_d, dtype=np.float64)
    rows_of = (lambda i: i) if id_of_row is None else id_of_row
    ex = exact_fp64(X, Q, np.where(gpu_ids >= 0, rows_of(np.maximum(gpu_ids, 0)), -1))
    checked = total = 0
    for b in range(B):
        k = int(K[b])
        gi, gd = gpu_ids[b, :k], gpu_d[b, :k]
        oi, od = ora_ids[b, :k], ora_d[b, :k]
        gv, ov = gi >= 0, oi >= 0
        assert len(set(gi[gv].tolist())) == gv.sum(), f"query {b}: duplicate ids"
        assert np.all(gv[:gv.sum()]), f"query {b}: padding before a result"
        assert np.all(np.diff(gd[gv]) >= 0), f"query {b}: distances not sorted"
        assert np.all(np.isinf(gd[~gv])), f"query {b}: padding distance"
        med = np.median(od[ov]) if ov.any() else 1.0
        tol = REL * np.maximum(ex[b, :k][gv], 1e-3 * med)
        err = np.abs(gd[gv].astype(np.float64) - ex[b, :k][gv])
        assert np.all(err <= tol), f"query {b}: distance error {err.max()} > {tol[np.argmax(err - tol)]}"
        no = int(ov.sum())
        total += no
        below = int(np.sum(od[:no] < amb_d[b]))
        if np.isinf(amb_d[b]):
            assert gv.sum() == no, f"query {b}: {gv.sum()} results vs oracle {no}"
        assert gv.sum() >= below, f"query {b}: {gv.sum()} results, oracle has {below} certain ones"
        for r in range(below):
            if not exact_ties:
                lo = r == 0 or od[r] - od[r - 1] > REL * od[r]
                hi = r == no - 1 or od[r + 1] - od[r] > REL * od[r + 1]
                if not (lo and hi):
                    continue
            assert gi[r] == oi[r], f"query {b} rank {r}: id {gi[r]} vs oracle {oi[r]} (amb_d {amb_d[b]})"
            if exact_ties:
                assert float(gd[r]) == od[r], f"query {b} rank {r}: distance {gd[r]} vs oracle {od[r]}"
            checked += 1
    assert checked >= min_checked * total, f"only {checked} of {total} oracle ranks checked"
    return checked, total


def recall(ids, gt, k):
    return float(np.mean([len(set(ids[b, :k].tolist()) & set(gt[b, :k].tolist())) / k
                          for b in range(len(ids))]))
