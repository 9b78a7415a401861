"""Pins of the oracle's OPQ-L pieces (Section V-B "Approximate Distances":
OPQ's asymmetric distance and the quantisation error as a third feature of
the learned correction): eigenvalue allocation worked by hand, encoding as
an argmin, the table-based asymmetric distance against the reconstruction,
the single test against a brute-force count, pruning off = exact, and the
three-feature fit's recall constraint."""
import numpy as np

from oracle import fit, ivf, pq, search


def test_eigen_allocation_scale_free_and_balanced():
    # the hand-worked example is tests/golden/opq_allocation_example.json;
    # a scale change of every variance changes nothing
    assert list(pq.eigen_allocation(np.array([8.0, 4.0, 2.0, 1.0]) * 1e-3, 2)) == [0, 3, 1, 2]
    # balance on a decaying spectrum: pairing the larger values of a round with
    # the smaller products never widens the spread of the log-products beyond
    # the widest round (here the first: var[0] / var[3])
    var = 1.0 / np.arange(1, 25)
    perm = pq.eigen_allocation(var, 4)
    assert sorted(perm.tolist()) == list(range(24))
    logs = [np.log(var[perm[j * 6:(j + 1) * 6]]).sum() for j in range(4)]
    assert max(logs) - min(logs) <= np.log(var[0] / var[3]) + 1e-12
    # every subspace gets one dim of each round
    rank = np.empty(24, int)
    rank[np.argsort(-var, kind="stable")] = np.arange(24)
    for j in range(4):
        assert sorted(rank[perm[j * 6:(j + 1) * 6]] // 4) == list(range(6))


def _small(seed=3, n=3000, D=16, m=4):
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((n, D)) * np.linspace(2.0, 0.3, D)).astype(np.float32)
    perm = pq.eigen_allocation(X.astype(np.float64).var(0), m)
    cb = pq.train_codebooks(X, perm, m, 4, np.arange(pq.KSUB))
    return X, perm, cb


def test_encode_is_the_nearest_centroid_and_adc_is_the_reconstruction_distance():
    X, perm, cb = _small()
    codes = pq.encode(X, perm, cb)
    m, _, ds = cb.shape
    for j in range(m):
        sub = X[:, perm[j * ds:(j + 1) * ds]].astype(np.float64)
        d = ((sub[:, None, :] - cb[j][None]) ** 2).sum(-1)
        assert np.all(d[np.arange(len(X)), codes[:, j]] <= d.min(1))
    rng = np.random.default_rng(9)
    Q = rng.standard_normal((5, X.shape[1]))
    T = pq.lut(Q, perm, cb)
    rec = pq.reconstruct(codes, perm, cb)
    for b in range(len(Q)):
        want = ((rec - Q[b]) ** 2).sum(1)
        assert np.allclose(pq.asymmetric_distance(T[b], codes), want, rtol=1e-12, atol=1e-12)
    e = pq.quantisation_error(X, codes, perm, cb)
    assert np.allclose(e, np.sqrt(((X - rec) ** 2).sum(1)), rtol=1e-12)


def _index_and_pq():
    X, perm, cb = _small(seed=5, n=2000)
    D = X.shape[1]
    rng = np.random.default_rng(2)
    C, a, _ = ivf.kmeans(X.astype(np.float64), rng.choice(len(X), 8, replace=False), 3)
    idx = search.OracleIndex(X, np.zeros(D), np.eye(D), C, a, dtype="f64")
    codes = pq.encode(idx.Xs, perm, cb)
    err = pq.quantisation_error(idx.Xs, codes, perm, cb)
    Q = (rng.standard_normal((12, D)) * np.linspace(2.0, 0.3, D)).astype(np.float32)
    return idx, Q, perm, cb, codes, err


def test_single_test_prunes_exactly_the_counted_candidates():
    idx, Q, perm, cb, codes, err = _index_and_pq()
    Qr = idx.rotate_queries(Q)
    T = pq.lut(Qr, perm, cb)
    pr = idx.probe(Qr, 3)
    tau = np.full(len(Q), 0.0)
    for b in range(len(Q)):
        tau[b] = np.sort(((idx.X - Q[b]) ** 2).sum(1))[40]
    m1, m3, beta = 0.9, -0.5, 0.2
    ids, d, st = search.search(idx, Q, pr, 3, 10, 16, None, None, mode="frozen", tau=tau, estimator="pq",
                               pq=dict(codes=codes, err=err, lut=T, m1=m1, m3=m3, beta=beta))
    for b in range(len(Q)):
        rows = np.concatenate([np.flatnonzero(idx.assign == l) for l in pr[b]])
        lhs = m1 * pq.asymmetric_distance(T[b], codes[rows]) + m3 * err[rows] + beta
        assert st[b, 0] == len(rows)
        assert st[b, 1] == int((lhs > tau[b]).sum())
        assert st[b, 2] == len(rows) - st[b, 1]
        assert st[b, 3] == st[b, 2] * idx.D       # a pruned candidate scans no rotated dimension


def test_disabled_classifier_is_pruning_off():
    idx, Q, perm, cb, codes, err = _index_and_pq()
    Qr = idx.rotate_queries(Q)
    T = pq.lut(Qr, perm, cb)
    pr = idx.probe(Qr, 4)
    S = search.n_steps(idx.D, 16)
    off = search.search(idx, Q, pr, 4, 10, 16, *search.disabled_tables(S))
    got = search.search(idx, Q, pr, 4, 10, 16, None, None, estimator="pq",
                        pq=dict(codes=codes, err=err, lut=T, m1=0.0, m3=0.0, beta=-np.inf))
    assert np.array_equal(got[0], off[0]) and np.array_equal(got[1], off[1])
    assert got[2][:, 1].sum() == 0


def test_three_feature_fit_keeps_label0_recall_and_uses_the_error():
    rng = np.random.default_rng(4)
    n = 4000
    tau = rng.uniform(1.0, 2.0, n)
    dis = rng.uniform(0.0, 4.0, n)
    err = rng.uniform(0.0, 1.0, n)
    # label 1 iff dis - 1.5 err > tau (a boundary that needs the error feature)
    lab = (dis - 1.5 * err > tau).astype(np.int8)
    m1, m3, bp, info = fit.fit_pq_correction(dis, err, tau, lab, r=0.99)
    assert info["enabled"] and info["grad"] < 1e-6
    keep0 = ~(m1 * dis[lab == 0] + m3 * err[lab == 0] + bp > tau[lab == 0])
    assert keep0.mean() >= 0.99
    # the fitted boundary leans on the error the way the labels do
    assert m3 < 0 and abs(m3 / m1 + 1.5) < 0.5
    pruned1 = (m1 * dis[lab == 1] + m3 * err[lab == 1] + bp > tau[lab == 1]).mean()
    assert pruned1 > 0.8


def test_encode_breaks_ties_to_the_lower_centroid():
    # two identical centroids in a subspace: the lower index wins every tie
    rng = np.random.default_rng(1)
    X = rng.standard_normal((50, 4))
    perm = np.arange(4)
    cb = rng.standard_normal((2, pq.KSUB, 2))
    cb[0, 7] = cb[0, 200] = [0.0, 0.0]        # a duplicate pair in subspace 0
    X[:, :2] = 0.0                             # every row is nearest to it
    codes = pq.encode(X, perm, cb)
    assert np.all(codes[:, 0] == 7)


def test_opq_rows_follow_the_classifier_on_every_stored_precision():
    # the single test reads the codes and errors it is given, whatever the
    # slab precision of the index (the estimate is the table, not the slab)
    X, perm, cb = _small(seed=8, n=1500)
    D = X.shape[1]
    rng = np.random.default_rng(3)
    C, a, _ = ivf.kmeans(X.astype(np.float64), rng.choice(len(X), 6, replace=False), 3)
    Q = (rng.standard_normal((5, D)) * np.linspace(2.0, 0.3, D)).astype(np.float32)
    out = []
    for dt in ("f32", "bf16"):
        idx = search.OracleIndex(X, np.zeros(D), np.eye(D), C, a, dtype=dt)
        codes = pq.encode(X.astype(np.float64), perm, cb)
        err = pq.quantisation_error(X.astype(np.float64), codes, perm, cb)
        T = pq.lut(idx.rotate_queries(Q), perm, cb)
        pr = idx.probe(idx.rotate_queries(Q), 3)
        out.append(search.search(idx, Q, pr, 3, 10, 16, None, None, estimator="pq",
                                 pq=dict(codes=codes, err=err, lut=T, m1=1.0, m3=-1.0, beta=0.0)))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][2], out[1][2])
