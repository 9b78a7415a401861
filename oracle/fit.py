"""Oracle data-driven distance correction, FP64 (Section V-A, V-B).

Section V-A recasts the error bound as a classifier: features dis' and tau,
label 1 when dis > tau (the candidate may be pruned) and label 0 otherwise;
a linear model sign(w1 dis' + w2 tau + b > 0) is rewritten as
m1 dis' + beta > tau.  "Adaptive Adjustment" then moves beta to a beta'
that reaches a target recall r on label 0.  "Incremental Correction"
(Section V-B) trains one classifier per Delta_d step.  Section VII-A sets
the labels (label 0 = the KNN of each training query, label 1 = up to 500k
samples collected while querying) and r = 0.995; the per-step target
r_s = 1 - (1 - r) / (D / Delta_d) appears in the paper's (commented)
parameter notes.

Readings where the paper is silent:
* Samples come from a replay of each training query with pruning off under
  the same tau schedule as search; a candidate tested against tau (finite)
  is label 0 if it is in the query's final exact top-K, label 1 if
  dis > tau, and dropped otherwise.
* Label-1 samples are thinned to at most ``cap`` by a counter-based draw:
  keep iff u < cap / n1 with u = SplitMix64-derived uniform of
  (seed, query, id) (Steele, Lea and Flood 2014).
* Features are scaled by the mean tau of the step's samples; the fit is a
  full-batch Newton (IRLS) logistic regression with ridge 1e-8 on the two
  weights, at most 50 iterations, stopping when max|gradient| < 1e-10.
* m1 = -w1 / w2 and beta = -b * tau_bar / w2, which needs w2 < 0; a step with
  w2 >= 0, fewer than 100 label-0 samples or no label-1 sample is disabled
  (m1 = 0, beta = -inf: never prunes).
* beta' is the largest value keeping label-0 recall >= r_s: with
  v_i = tau_i - m1 * dis'_i over the label-0 samples sorted ascending and
  f = floor((1 - r_s) * n0), beta' = v_(f+1); the test prunes iff
  beta' > v.  The bisection the paper describes reaches the same value.
* Step s is trained on the samples that no earlier step pruned.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied to a counter (uint64, wraps)."""
    with np.errstate(over="ignore"):
        z = np.asarray(z, dtype=np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def sample_uniform(seed: int, query: np.ndarray, ids: np.ndarray) -> np.ndarray:
    """u in [0, 1): 53 high bits of splitmix64(seed ^ splitmix64((query << 32) ^ id))."""
    key = (np.asarray(query, dtype=np.uint64) << np.uint64(32)) ^ np.asarray(ids).astype(np.uint64)
    z = splitmix64(np.uint64(seed) ^ splitmix64(key))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def label_rows(rows: dict, topk_ids: np.ndarray, seed: int = 0, cap: int = 500_000, keys: bool = False):
    """Label replay rows; returns (partials, tau, label) of the kept rows
    (with keys: also their query index and candidate id)."""
    tau, dis = rows["tau"], rows["dis"]
    finite = np.isfinite(tau)
    in_top = (np.asarray(topk_ids)[rows["query"]] == rows["id"][:, None]).any(axis=1)
    lab0 = finite & in_top
    lab1 = finite & ~in_top & (dis > tau)
    n1 = int(lab1.sum())
    if n1 > cap:
        u = sample_uniform(seed, rows["query"], rows["id"])
        lab1 &= u < cap / n1
    keep = lab0 | lab1
    if keys:
        return rows["partials"][keep], tau[keep], lab1[keep].astype(np.int8), rows["query"][keep], rows["id"][keep]
    return rows["partials"][keep], tau[keep], lab1[keep].astype(np.int8)


def _loss_grad(theta, A, y, ridge):
    k = len(theta) - 1
    z = A @ theta
    # log(1 + e^z) - y z, computed stably
    loss = np.mean(np.logaddexp(0.0, z) - y * z) + 0.5 * ridge * float(theta[:k] @ theta[:k])
    p = 0.5 * (1.0 + np.tanh(0.5 * z))
    g = A.T @ (p - y) / len(y)
    g[:k] += ridge * theta[:k]
    return loss, g, p


def fit_logistic(F: np.ndarray, y: np.ndarray, ridge: float = 1e-8, max_iter: int = 50,
                 tol: float = 1e-10):
    """Minimise mean binary cross-entropy + ridge/2 * |w|^2 of
    P(y = 1) = sigmoid(w . f + b) by damped Newton steps (any number of
    features; the correction of Section V-A uses f = (dis', tau), OPQ-L adds
    the quantisation error).  Returns (theta = [w..., b], iterations,
    max |gradient|)."""
    A = np.column_stack([np.asarray(F, dtype=np.float64), np.ones(len(y))])
    y = np.asarray(y, dtype=np.float64)
    k = A.shape[1] - 1
    theta = np.zeros(k + 1)
    loss, g, p = _loss_grad(theta, A, y, ridge)
    it = 0
    for it in range(1, max_iter + 1):
        if np.max(np.abs(g)) < tol:
            it -= 1
            break
        w = p * (1.0 - p) / len(y)
        H = A.T @ (A * w[:, None])
        H[np.arange(k), np.arange(k)] += ridge
        step = np.linalg.solve(H, g)
        t = 1.0
        while True:
            cand = theta - t * step
            l2, g2, p2 = _loss_grad(cand, A, y, ridge)
            # near the optimum the loss change is below rounding; a step that
            # shrinks the gradient is accepted then
            if l2 <= loss or np.max(np.abs(g2)) < np.max(np.abs(g)) or t < 1e-10:
                break
            t *= 0.5
        theta, loss, g, p = cand, l2, g2, p2
    return theta, it, float(np.max(np.abs(g)))


def beta_prime_closed_form(v0: np.ndarray, r_s: float) -> float:
    """Largest beta with #{v < beta} <= floor((1 - r_s) n0): v_(f+1)."""
    v = np.sort(np.asarray(v0, dtype=np.float64))
    f = int(math.floor((1.0 - r_s) * len(v)))
    return float(v[min(f, len(v) - 1)])


def beta_prime_bisection(v0: np.ndarray, r_s: float) -> float:
    """The paper's binary search for beta': bisect on beta until the
    bracket [lo, hi] is one ulp wide; lo keeps recall >= r_s, hi does not."""
    v = np.asarray(v0, dtype=np.float64)
    n0 = len(v)

    def ok(beta):
        return 1.0 - np.count_nonzero(v < beta) / n0 >= r_s

    lo = float(v.min())
    hi = float(v.max())
    if ok(np.nextafter(hi, np.inf)):
        return float(np.nextafter(hi, np.inf))
    hi = float(np.nextafter(hi, np.inf))
    while np.nextafter(lo, np.inf) < hi:
        mid = lo + (hi - lo) / 2.0
        if mid <= lo or mid >= hi:
            mid = float(np.nextafter(lo, np.inf))
        if ok(mid):
            lo = mid
        else:
            hi = mid
    return lo


def fit_correction(partials: np.ndarray, tau: np.ndarray, label: np.ndarray, D: int,
                   delta_d: int, r: float = 0.995, min_label0: int = 100):
    """Sequential per-step fit.  Returns (m1[S-1], beta'[S-1], info list)."""
    S = -(-D // delta_d)
    r_s = 1.0 - (1.0 - r) / S
    n = len(tau)
    active = np.ones(n, dtype=bool)
    lab0 = np.asarray(label) == 0
    m1 = np.zeros(max(S - 1, 0))
    beta = np.full(max(S - 1, 0), -np.inf)
    info = []
    for s in range(1, S):
        a = active
        p = partials[:, s - 1]
        n0 = int((a & lab0).sum())
        n1 = int((a & ~lab0).sum())
        rec = dict(step=s, n0=n0, n1=n1, enabled=False)
        if n0 >= min_label0 and n1 > 0:
            tb = float(tau[a].mean())
            F = np.column_stack([p[a] / tb, tau[a] / tb])
            theta, iters, gmax = fit_logistic(F, (~lab0[a]).astype(np.float64))
            w1, w2, b = theta
            rec.update(w1=w1, w2=w2, b=b, tau_bar=tb, iters=iters, grad=gmax)
            if w2 < 0:
                m = -w1 / w2
                v = tau[a & lab0] - m * p[a & lab0]
                bp = beta_prime_closed_form(v, r_s)
                m1[s - 1] = m
                beta[s - 1] = bp
                rec.update(enabled=True, m1=m, beta=-b * tb / w2, beta_prime=bp)
                active = active & ~(m * p + bp > tau)
        info.append(rec)
    return m1, beta, info


def fit_pq_correction(dis: np.ndarray, err: np.ndarray, tau: np.ndarray, label: np.ndarray, r: float = 0.995,
                      min_label0: int = 100):
    """OPQ-L's classifier (Section V-B "Approximate Distances": features the
    asymmetric distance dis', the threshold tau and the distance e from the
    vector to its quantised reconstruction; one classifier, no steps).
    Logistic fit on (dis'/tau_bar, tau/tau_bar, e/sqrt(tau_bar)) as above;
    prune iff m1 dis' + m3 e + beta > tau with m1 = -w1/w2,
    m3 = -w3 sqrt(tau_bar)/w2; beta' is the largest value keeping label-0
    recall >= r (v_i = tau_i - m1 dis'_i - m3 e_i over label 0, the
    (floor((1 - r) n0) + 1)-th smallest).  Returns (m1, m3, beta', info);
    a failed fit (w2 >= 0, too few samples) returns (0, 0, -inf)."""
    dis = np.asarray(dis, dtype=np.float64)
    err = np.asarray(err, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64)
    lab0 = np.asarray(label) == 0
    n0, n1 = int(lab0.sum()), int((~lab0).sum())
    info = dict(n0=n0, n1=n1, enabled=False)
    if n0 < min_label0 or n1 == 0:
        return 0.0, 0.0, -np.inf, info
    tb = float(tau.mean())
    F = np.column_stack([dis / tb, tau / tb, err / math.sqrt(tb)])
    theta, iters, gmax = fit_logistic(F, (~lab0).astype(np.float64))
    w1, w2, w3, b = theta
    info.update(w1=w1, w2=w2, w3=w3, b=b, tau_bar=tb, iters=iters, grad=gmax)
    if not w2 < 0:
        return 0.0, 0.0, -np.inf, info
    m1 = -w1 / w2
    m3 = -w3 * math.sqrt(tb) / w2
    v = tau[lab0] - m1 * dis[lab0] - m3 * err[lab0]
    bp = beta_prime_closed_form(v, r)
    info.update(enabled=True, m1=m1, m3=m3, beta=-b * tb / w2, beta_prime=bp)
    return m1, m3, bp, info
