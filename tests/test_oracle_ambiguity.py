"""Pins of the oracle's ambiguity bookkeeping (the rule the GPU parity tests
rely on to compare ids rank by rank).

The oracle marks a candidate uncertain when another rounding of the same
arithmetic could decide it otherwise, for any tau the other side can hold
once earlier uncertain decisions went the other way; amb_d is the smallest
exact distance of an uncertain candidate.  Claim: any other run whose
decisions stay within the rounding model returns, below amb_d, exactly the
oracle's entries.  The pins plant such another run -- the same oracle on
stored values moved to the edges of their deviation bounds (Xdev) at random
coordinates -- and check the claim, including through the tau cascade of
later waves.
"""
import copy

import numpy as np
import pytest

import synth
from oracle import fit, ivf, pca, search, storage


@pytest.fixture(scope="module")
def bf16_setup():
    X, Q, T, cfg = synth.workload("tiny", n_train=400)
    mu, R, _ = pca.train_rotation(X)
    Xr = pca.rotate(X, mu, R)
    init = np.random.default_rng(7).choice(len(X), cfg["nlist"], replace=False)
    C, a, _ = ivf.kmeans(Xr, init, 6)
    # a large rotation slack (1e-3 of the norm) makes many coordinates
    # flippable, so the planted runs disagree often
    oidx = search.OracleIndex(X, mu, R, C, a, dtype="bf16", flip_eps=1e-3)
    pr_t = oidx.probe(oidx.rotate_queries(T), 8)
    rows = search.collect(oidx, T, pr_t, 8, 10, 16)
    top, _, _ = search.search(oidx, T, pr_t, 8, 10, 16, *search.disabled_tables(8))
    P, tau, lab = fit.label_rows(rows, top, cap=100_000)
    m1, beta, _ = fit.fit_correction(P, tau, lab, 128, 16, r=0.99, min_label0=20)
    pr = oidx.probe(oidx.rotate_queries(Q), 16)
    return dict(oidx=oidx, Q=Q, pr=pr, m1=m1, beta=beta, Xr=Xr)


def _planted(oidx, seed):
    """The oracle index with every stored coordinate moved by -Xdev, 0 or
    +Xdev (equally likely): another implementation within the model."""
    o2 = copy.copy(oidx)
    u = np.random.default_rng(seed).integers(-1, 2, size=oidx.Xs.shape)
    o2.Xs = oidx.Xs + u * oidx.Xdev
    o2.Xdev = None
    return o2


def _agree_below(ids_a, d_a, ids_b, d_b, amb_d):
    """Ranks with an entry below amb_d: same (id, distance); returns the
    number of such ranks."""
    n = 0
    for b in range(ids_a.shape[0]):
        below = np.isfinite(d_a[b]) & (d_a[b] < amb_d[b])
        k = int(below.sum())
        assert np.all(below[:k]), "entries below amb_d form a prefix"
        assert np.array_equal(ids_a[b, :k], ids_b[b, :k]), f"query {b}"
        assert np.array_equal(d_a[b, :k], d_b[b, :k]), f"query {b}"
        n += k
    return n


@pytest.mark.parametrize("mode,fw,g,bites", [("waves", 1, 1, True), ("waves", 2, 2, True), ("waves", 4, 30, False),
                                             ("sequential", 1, 1, True)])
def test_planted_rounding_agrees_below_amb_d(bf16_setup, mode, fw, g, bites):
    s = bf16_setup
    kw = dict(mode=mode, first_wave=fw, growth=g)
    ids, d, st, amb_d = search.search(s["oidx"], s["Q"], s["pr"], 16, 10, 16, s["m1"], s["beta"], with_amb=True,
                                      **kw)
    assert st[:, 4].sum() > 0 and np.isfinite(amb_d).any()
    differ = 0
    checked = 0
    for seed in range(6):
        o2 = _planted(s["oidx"], seed)
        i2, d2, st2 = search.search(o2, s["Q"], s["pr"], 16, 10, 16, s["m1"], s["beta"], **kw)
        checked += _agree_below(ids, d, i2, d2, amb_d)
        differ += int((i2 != ids).any(axis=1).sum())
        # candidates never marked uncertain are decided alike: equal work
        # counters on queries without any uncertain candidate
        un = st[:, 4] == 0
        assert np.array_equal(st[un, :4], st2[un, :4])
    # with many waves the planted runs really return other results (beyond
    # amb_d), and most ranks are checked
    assert differ > 0 or not bites
    assert checked > 0.5 * 6 * np.isfinite(d).sum()


def test_planted_rotation_errors_agree_below_amb_d():
    """FP32 slabs and a rotation that may differ per coordinate by
    flip_eps * ||x'|| on the database and qdev_eps * ||q'|| on the queries:
    a run whose rotated values sit anywhere in those ranges agrees below
    amb_d, through several waves."""
    X, Q, T, cfg = synth.workload("tiny", n_train=300)
    mu, R, _ = pca.train_rotation(X)
    Xr = pca.rotate(X, mu, R)
    init = np.random.default_rng(7).choice(len(X), cfg["nlist"], replace=False)
    C, a, _ = ivf.kmeans(Xr, init, 6)
    eps = 3e-3
    oidx = search.OracleIndex(X, mu, R, C, a, dtype="f32", flip_eps=eps)
    pr_t = oidx.probe(oidx.rotate_queries(T), 8)
    rows = search.collect(oidx, T, pr_t, 8, 10, 16)
    top, _, _ = search.search(oidx, T, pr_t, 8, 10, 16, *search.disabled_tables(8))
    P, tau, lab = fit.label_rows(rows, top, cap=100_000)
    m1, beta, _ = fit.fit_correction(P, tau, lab, 128, 16, r=0.99, min_label0=20)
    pr = oidx.probe(oidx.rotate_queries(Q), 16)
    ids, d, st, amb_d = search.search(oidx, Q, pr, 16, 10, 16, m1, beta, first_wave=1, growth=1, with_amb=True,
                                      qdev_eps=eps)
    Qr = oidx.rotate_queries(Q)
    qd = eps * np.linalg.norm(Qr, axis=1, keepdims=True)
    differ = checked = 0
    for seed in range(4):
        rng = np.random.default_rng(100 + seed)
        o2 = _planted(oidx, seed)
        shift = rng.uniform(-1, 1, size=Qr.shape) * qd
        o2.rotate_queries = (lambda M, base=oidx.rotate_queries, sh=shift: base(M) + sh)
        i2, d2, _ = search.search(o2, Q, pr, 16, 10, 16, m1, beta, first_wave=1, growth=1)
        checked += _agree_below(ids, d, i2, d2, amb_d)
        differ += int((i2 != ids).any(axis=1).sum())
    # the planted runs return other results beyond amb_d, and the check is
    # not vacuous (at this stress level about half of the ranks are certain)
    assert differ > 0
    assert checked > 0.3 * 4 * np.isfinite(d).sum()


def test_no_band_no_flips_means_nothing_uncertain():
    X, Q, T, cfg = synth.workload("tiny", n_train=200)
    mu, R, _ = pca.train_rotation(X)
    Xr = pca.rotate(X, mu, R)
    init = np.random.default_rng(7).choice(len(X), cfg["nlist"], replace=False)
    C, a, _ = ivf.kmeans(Xr, init, 4)
    oidx = search.OracleIndex(X, mu, R, C, a, dtype="f32")
    pr = oidx.probe(oidx.rotate_queries(Q), 8)
    S = search.n_steps(128, 16)
    # exact-safe tables (prune iff dis' > tau): continuous data, no band
    ids, d, st, amb_d = search.search(oidx, Q, pr, 8, 10, 16, np.ones(S - 1), np.zeros(S - 1), first_wave=1,
                                      with_amb=True)
    assert st[:, 4].sum() == 0 and np.all(np.isinf(amb_d))
    # a band makes decisions near tau uncertain, and amb_d is then the exact
    # distance of one of them: no smaller than tau at the test, so with the
    # exact-safe tables (dis' <= dis) never below the final K-th distance
    ids, d, st, amb_d = search.search(oidx, Q, pr, 8, 10, 16, np.ones(S - 1), np.zeros(S - 1), first_wave=1,
                                      amb=0.05, with_amb=True)
    assert st[:, 4].sum() > 0
    fin = np.isfinite(amb_d)
    assert np.all(amb_d[fin] >= d[fin, 9] * (1 - 0.05))


def test_deviation_bound_is_the_neighbouring_rounding():
    """With a rotation slack e below half a unit of the format, Xdev is
    nonzero exactly at the coordinates whose exact value lies within e of a
    rounding midpoint, and there it is one unit (the neighbouring value on
    the other side of that midpoint)."""
    rng = np.random.default_rng(3)
    # magnitudes in [0.5, 1): one BF16 unit is 2^-8 there
    X = (rng.uniform(0.5, 1.0, size=(500, 32)) * rng.choice([-1.0, 1.0], size=(500, 32))).astype(np.float32)
    mu, R = np.zeros(32), np.eye(32)
    C = X[:4].astype(np.float64)
    a = np.zeros(500, np.int32)
    eps = 2e-4  # e = eps * ||x|| < 2e-4 * sqrt(32) < 2^-9
    oidx = search.OracleIndex(X, mu, R, C, a, dtype="bf16", flip_eps=eps)
    x = X.astype(np.float64)
    e = eps * np.linalg.norm(x, axis=1, keepdims=True)
    assert e.max() < 2.0 ** -9
    unit = 2.0 ** -8
    # distance of |x| to the nearest midpoint k*unit + unit/2 of the BF16 grid
    t = np.abs(x) / unit - 0.5
    to_mid = np.abs(t - np.round(t)) * unit
    near = to_mid <= e
    dev = oidx.Xdev
    assert near.any() and not near.all()
    assert np.array_equal(dev > 0, near)
    assert np.allclose(dev[near], unit, rtol=0, atol=1e-12)


def test_fp8_deviation_bound_covers_a_moved_scale():
    """FP8: the per-dimension scale amax / 448 moves when the column maximum
    does; Xdev covers the stored values under any scale within that range."""
    rng = np.random.default_rng(4)
    X = rng.normal(size=(400, 16)).astype(np.float32)
    mu, R = np.zeros(16), np.eye(16)
    C = X[:4].astype(np.float64)
    a = np.zeros(400, np.int32)
    eps = 1e-5
    oidx = search.OracleIndex(X, mu, R, C, a, dtype="fp8", flip_eps=eps)
    x = X.astype(np.float64)
    s = storage.fp8_scales(storage.to_fp32(x)).astype(np.float64)
    e_max = eps * np.linalg.norm(x, axis=1).max()
    for f in (1 - e_max / (448 * s), 1 + e_max / (448 * s)):
        moved = storage.stored(x, "fp8", (s * f).astype(np.float32))
        assert np.all(np.abs(moved - oidx.Xs) <= oidx.Xdev * (1 + 1e-9) + 1e-12)
    assert np.all(oidx.Xdev > 0)  # every value moves with its scale
