"""Pins of the oracle refinement loop (Section I result queue, Algorithm 2 loop
structure, Section V-A/B learned test and incremental correction)."""
import numpy as np
import pytest

from oracle import ivf, knn, pca, search


def _worked_index(order_b=(3, 2, 4)):
    # D = 4, Delta_d = 2 (S = 2: one test after two dims, then the exact
    # distance), identity rotation, query at the origin, K = 2.
    X = np.array([[1, 0, 1, 0],   # id 0: dis'_1 = 1, dis = 2
                  [0, 2, 0, 0],   # id 1: dis'_1 = 4, dis = 4
                  [1, 1, 0, 3],   # id 2: dis'_1 = 2, dis = 11
                  [0, 1, 1, 1],   # id 3: dis'_1 = 1, dis = 3
                  [2, 0, 0, 0]],  # id 4: dis'_1 = 4, dis = 4
                 dtype=np.float32)
    assign = np.array([0, 0, 1, 1, 1], dtype=np.int32)
    idx = search.OracleIndex(X, np.zeros(4), np.eye(4), np.zeros((2, 4)), assign, dtype="f64")
    # storage order inside list 1 chosen by the caller (3, 2, 4 by default)
    idx.members = np.array([0, 1] + list(order_b), dtype=np.int64)
    return idx


def test_worked_example_ties_and_padding():
    # ids 1 and 4 are both at distance 4: with K = 3 and no pruning the third
    # entry is id 1 (lower id wins the tie); with K = 7 the tail is padded.
    idx = _worked_index(order_b=(4, 3, 2))
    Q = np.zeros((1, 4), dtype=np.float32)
    m1, beta = search.disabled_tables(2)
    ids, d, _ = search.search(idx, Q, np.array([[1, 0]], np.int32), 2, 3, 2, m1, beta,
                              mode="sequential")
    assert list(ids[0]) == [0, 3, 1] and list(d[0]) == [2, 3, 4]
    ids, d, _ = search.search(idx, Q, np.array([[0, 1]], np.int32), 2, 7, 2, m1, beta)
    assert list(ids[0]) == [0, 3, 1, 4, 2, -1, -1]
    assert list(d[0][:5]) == [2, 3, 4, 4, 11] and np.all(np.isinf(d[0][5:]))


@pytest.fixture(scope="module")
def small():
    rng = np.random.default_rng(21)
    D, N, nlist = 24, 3000, 12
    X = (rng.standard_normal((N, D)) * np.linspace(3, 0.2, D)).astype(np.float32)
    centers = X[rng.choice(N, nlist, replace=False)].astype(np.float64)
    C, a, _ = ivf.kmeans(X.astype(np.float64), np.arange(nlist), 4)
    a = ivf.assign(X.astype(np.float64), C)
    del centers
    Q = (rng.standard_normal((40, D)) * np.linspace(3, 0.2, D)).astype(np.float32)
    idx = search.OracleIndex(X, np.zeros(D), np.eye(D), C, a, dtype="f64")
    return dict(X=X, Q=Q, idx=idx, D=D, nlist=nlist)


def _probed_brute_force(idx, Q, probes, K):
    out = []
    for b in range(len(Q)):
        cand = np.concatenate([idx.members[idx.list_off[l]:idx.list_off[l + 1]] for l in probes[b]])
        d = ((idx.X[cand].astype(np.float64) - Q[b].astype(np.float64)) ** 2).sum(1)
        o = np.lexsort((cand, d))[:K]
        out.append((cand[o], d[o]))
    return out


@pytest.mark.parametrize("mode", ["sequential", "waves"])
def test_pruning_off_equals_brute_force_over_probed_candidates(small, mode):
    idx, Q = small["idx"], small["Q"]
    probes = idx.probe(idx.rotate_queries(Q), 4)
    m1, beta = search.disabled_tables(search.n_steps(small["D"], 8))
    ids, d, st = search.search(idx, Q, probes, 4, 10, 8, m1, beta, mode=mode, final_rel=np.inf)
    for b, (ri, rd) in enumerate(_probed_brute_force(idx, Q, probes, 10)):
        # FP64 sums in another order: equal up to rounding
        assert np.array_equal(ids[b], ri) and np.allclose(d[b], rd, rtol=1e-13, atol=0)
    assert np.all(st[:, 1] == 0) and np.all(st[:, 2] == st[:, 0])
    # with the test on the completed distance: same result, fewer exact distances
    ids2, d2, st2 = search.search(idx, Q, probes, 4, 10, 8, m1, beta, mode=mode, final_rel=search.FINAL_REL)
    assert np.array_equal(ids2, ids) and np.array_equal(d2, d)
    assert st2[:, 2].sum() < st[:, 2].sum()
    assert np.array_equal(st2[:, 3], st[:, 3])  # pruned at d = D still scanned D dims


def test_all_lists_probed_equals_exact_knn(small):
    idx, Q = small["idx"], small["Q"]
    probes = idx.probe(idx.rotate_queries(Q), small["nlist"])
    m1, beta = search.disabled_tables(search.n_steps(small["D"], 8))
    ids, d, _ = search.search(idx, Q, probes, small["nlist"], 10, 8, m1, beta)
    gi, gd = knn.exact_knn(small["X"], Q, 10)
    assert np.array_equal(ids, gi) and np.allclose(d, gd, rtol=1e-13, atol=0)


def test_exact_safe_tables_match_pruning_off_for_every_schedule(small):
    # m1 = 1, beta = 0 prunes iff dis'_s > tau.  dis'_s <= dis (a partial sum
    # of the same non-negative terms after an orthogonal rotation) and every
    # schedule's tau is >= the final K-th distance, so nothing in the final
    # result is ever pruned.
    idx, Q = small["idx"], small["Q"]
    probes = idx.probe(idx.rotate_queries(Q), 6)
    S = search.n_steps(small["D"], 8)
    off = search.disabled_tables(S)
    safe = (np.ones(S - 1), np.zeros(S - 1))
    ref_ids, ref_d, _ = search.search(idx, Q, probes, 6, 10, 8, *off)
    for mode, fw, g in [("sequential", 1, 1), ("waves", 1, 1), ("waves", 2, 1), ("waves", 6, 1),
                        ("waves", 1, 2), ("waves", 2, 30)]:
        ids, d, st = search.search(idx, Q, probes, 6, 10, 8, *safe, mode=mode, first_wave=fw, growth=g)
        assert np.array_equal(ids, ref_ids) and np.array_equal(d, ref_d)
    ids, d, st = search.search(idx, Q, probes, 6, 10, 8, *safe, mode="frozen", tau=ref_d[:, -1])
    assert np.array_equal(ids, ref_ids) and np.array_equal(d, ref_d)
    assert st[:, 1].sum() > 0  # and it does prune


def test_containment_of_unprunable_true_neighbours(small):
    # tau under any schedule is >= tau_F (final K-th distance); the test is
    # monotone in tau, so every exact top-K member that survives a frozen
    # test at tau_F is returned by every schedule.
    idx, Q = small["idx"], small["Q"]
    probes = idx.probe(idx.rotate_queries(Q), 6)
    S = search.n_steps(small["D"], 8)
    aggressive = (np.full(S - 1, 1.6), np.full(S - 1, 2.0))
    ref_ids, ref_d, _ = search.search(idx, Q, probes, 6, 10, 8, *search.disabled_tables(S))
    fz_ids, _, _ = search.search(idx, Q, probes, 6, 10, 8, *aggressive, mode="frozen",
                                 tau=ref_d[:, -1])
    for mode in ["sequential", "waves"]:
        ids, _, st = search.search(idx, Q, probes, 6, 10, 8, *aggressive, mode=mode)
        assert st[:, 1].sum() > 0
        for b in range(len(Q)):
            A = set(ref_ids[b]) & set(fz_ids[b][fz_ids[b] >= 0])
            assert A <= set(ids[b])


def test_partial_distances_monotone_lower_bounds(small):
    idx, Q = small["idx"], small["Q"]
    probes = idx.probe(idx.rotate_queries(Q[:10]), 3)
    rows = search.collect(idx, Q[:10], probes, 3, 10, 8)
    P = rows["partials"]
    assert np.all(np.diff(P, axis=1) >= 0)
    assert np.all(P[:, -1] <= rows["dis"] * (1 + 1e-12) + 1e-12)
    # adding the last slab closes the gap exactly (f64 storage, identity R)
    last = ((idx.Xs[np.searchsorted(idx.ids, rows["id"])][:, 16:] -
             idx.rotate_queries(Q[:10])[rows["query"]][:, 16:]) ** 2).sum(1)
    assert np.allclose(P[:, -1] + last, rows["dis"], rtol=1e-12, atol=1e-12)


def test_wave_bounds_growth():
    assert search.wave_bounds(64, 1, 1) == [0, 1, 2, 4, 8, 16, 32, 64]
    assert search.wave_bounds(64, 8, 2) == [0, 8, 32, 64]
    assert search.wave_bounds(64, 8, 30) == [0, 8, 64]
    assert search.wave_bounds(5, 8, 1) == [0, 5]


def test_collect_tau_is_the_waves_schedule_tau(small):
    idx, Q = small["idx"], small["Q"]
    probes = idx.probe(idx.rotate_queries(Q[:5]), 5)
    rows = search.collect(idx, Q[:5], probes, 5, 10, 8, first_wave=1)
    for b in range(5):
        r = rows["query"] == b
        n0 = idx.list_off[probes[b, 0] + 1] - idx.list_off[probes[b, 0]]
        tb = rows["tau"][r]
        assert np.all(np.isinf(tb[:n0]))
        if n0 >= 10:
            assert tb[n0] == np.sort(rows["dis"][r][:n0])[9]


def test_rotation_invariance_of_results(small):
    # An orthogonal rotation changes partial distances but not exact ones:
    # with pruning off the result is the same under any rotation.
    idx0, Q = small["idx"], small["Q"]
    rng = np.random.default_rng(8)
    Rq, _ = np.linalg.qr(rng.standard_normal((small["D"], small["D"])))
    mu = rng.standard_normal(small["D"])
    idx1 = search.OracleIndex(small["X"], mu, Rq, (idx0.C - 0) @ Rq.T - mu @ Rq.T,
                              idx0.assign, dtype="f64")
    probes = idx0.probe(idx0.rotate_queries(Q), 4)
    S = search.n_steps(small["D"], 8)
    a = search.search(idx0, Q, probes, 4, 10, 8, *search.disabled_tables(S))
    b = search.search(idx1, Q, probes, 4, 10, 8, *search.disabled_tables(S))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_integer_data_gives_integer_distances():
    rng = np.random.default_rng(2)
    X = rng.integers(0, 256, size=(500, 16)).astype(np.float32)
    Q = rng.integers(0, 256, size=(4, 16)).astype(np.float32)
    idx = search.OracleIndex(X, np.zeros(16), np.eye(16), np.zeros((1, 16)),
                             np.zeros(500, np.int32))
    ids, d, _ = search.search(idx, Q, np.zeros((4, 1), np.int32), 1, 20, 8,
                              *search.disabled_tables(2))
    assert np.all(d == np.rint(d)) and np.all(d < 2 ** 24)


@pytest.fixture(scope="module")
def rotated():
    """PCA-rotated small set stored in every slab precision."""
    rng = np.random.default_rng(23)
    D, N, nlist = 32, 4000, 16
    X = np.rint((rng.standard_normal((N, D)) * np.linspace(40, 3, D)) + 100).astype(np.float32)
    Q = np.rint((rng.standard_normal((30, D)) * np.linspace(40, 3, D)) + 100).astype(np.float32)
    from oracle import pca
    mu, Rm, _ = pca.train_rotation(X)
    Xr = pca.rotate(X, mu, Rm)
    C, _, _ = ivf.kmeans(Xr, np.arange(nlist), 4)
    a = ivf.assign(Xr, C)
    idx = {dt: search.OracleIndex(X, mu, Rm, C, a, dtype=dt) for dt in ("f32", "bf16", "fp8")}
    return dict(X=X, Q=Q, idx=idx, D=D, nlist=nlist, Xr=Xr)


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_quantisation_error_bound_holds_for_every_pair(rotated, dtype):
    # ||q' - x~|| <= ||q' - x'|| + ||x' - x~|| (triangle inequality), so a
    # candidate whose rotated distance is <= tau has dis'_S <= (sqrt(tau) + e_x)^2.
    idx = rotated["idx"][dtype]
    Qr = idx.rotate_queries(rotated["Q"])
    assert np.all(idx.xerr > 0)
    ps = ((Qr[:, None, :] - idx.Xs[None, :, :]) ** 2).sum(-1)
    dr = ((Qr[:, None, :] - rotated["Xr"][None, :, :]) ** 2).sum(-1)
    bound = (np.sqrt(dr) + idx.xerr[None, :]) ** 2
    assert np.all(ps <= bound * (1 + 1e-12))
    # and e_x is no larger than it must be: some pair uses most of the slack
    assert np.max((ps - dr) / (bound - dr)) > 0.5
    assert np.array_equal(rotated["idx"]["f32"].xerr, np.zeros(len(rotated["X"])))


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_final_test_never_changes_the_result(rotated, dtype):
    # It drops only candidates whose exact distance exceeds tau, which could
    # not enter the result queue: results are identical with and without it,
    # under every schedule, with the learned tests on or off.
    idx, Q = rotated["idx"][dtype], rotated["Q"]
    probes = idx.probe(idx.rotate_queries(Q), 6)
    S = search.n_steps(rotated["D"], 8)
    tabs = [search.disabled_tables(S), (np.full(S - 1, 1.3), np.full(S - 1, 50.0))]
    for m1, beta in tabs:
        for mode, fw, g in [("sequential", 1, 1), ("waves", 1, 1), ("waves", 2, 30)]:
            a = search.search(idx, Q, probes, 6, 10, 8, m1, beta, mode=mode, first_wave=fw, growth=g,
                              final_rel=np.inf)
            b = search.search(idx, Q, probes, 6, 10, 8, m1, beta, mode=mode, first_wave=fw, growth=g,
                              final_rel=search.FINAL_REL)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), (mode, fw, g)
            assert b[2][:, 2].sum() <= a[2][:, 2].sum()
            if not np.any(m1):  # learned tests off: the final test is the only one
                assert b[2][:, 2].sum() < a[2][:, 2].sum()


def test_res_estimate_is_exact_for_a_query_at_the_origin(small):
    # q = 0: ||q_r||^2 = 0 and sigma = 0, so C1 - C2 = ||x||^2 = dis at every
    # step and RES prunes exactly the candidates with dis > tau: the results
    # equal the pruning-off results, and every exact distance taken is <= tau
    idx = small["idx"]
    Q = np.zeros((1, small["D"]), np.float32)
    probes = idx.probe(idx.rotate_queries(Q), small["nlist"])
    S = search.n_steps(small["D"], 8)
    off = search.search(idx, Q, probes, small["nlist"], 10, 8, *search.disabled_tables(S))
    res = search.search(idx, Q, probes, small["nlist"], 10, 8, None, None, estimator="res", res_m=8.0,
                        mode="sequential")
    assert np.array_equal(res[0], off[0]) and np.allclose(res[1], off[1], rtol=1e-13)
    assert res[2][0, 1] > 0 and res[2][0, 1] + res[2][0, 2] == res[2][0, 0]


@pytest.mark.parametrize("m", [0.5, 1.0, 2.0])
def test_res_loss_rate_follows_the_gaussian_error_model(m):
    # x ~ N(0, diag(lam)) (already rotated), so for a query q the error
    # C1 - C2 - dis = 2 <q_r, x_r> ~ N(0, sigma^2) exactly (Eq. 2).  With a
    # frozen tau just above a candidate's distance, the candidate is lost iff
    # that error exceeds m sigma: probability 1 - Phi(m).
    from math import erf, sqrt
    rng = np.random.default_rng(5)
    D, N = 32, 20000
    lam = np.linspace(4.0, 0.2, D)
    X = (rng.standard_normal((N, D)) * np.sqrt(lam)).astype(np.float32)
    Q = (rng.standard_normal((400, D)) * np.sqrt(lam)).astype(np.float32)
    idx = search.OracleIndex(X, np.zeros(D), np.eye(D), np.zeros((1, D)), np.zeros(N, np.int32), dtype="f64")
    # one query per candidate: tau = that candidate's distance (+ a hair)
    cand = rng.choice(N, len(Q), replace=False)
    dis = ((X[cand].astype(np.float64) - Q.astype(np.float64)) ** 2).sum(1)
    lost = 0
    for b in range(len(Q)):
        one = search.OracleIndex(X[cand[b:b + 1]], np.zeros(D), np.eye(D), np.zeros((1, D)), np.zeros(1, np.int32),
                                 dtype="f64", ids=cand[b:b + 1])
        one.var = idx.var  # sigma_i^2 of the whole population
        ids, _, _ = search.search(one, Q[b:b + 1], np.zeros((1, 1), np.int32), 1, 1, 16, None, None,
                                  mode="frozen", tau=np.array([dis[b] * (1 + 1e-12)]), estimator="res", res_m=m)
        lost += ids[0, 0] < 0
    want = 1 - 0.5 * (1 + erf(m / sqrt(2)))
    got = lost / len(Q)
    assert abs(got - want) < 4 * sqrt(want * (1 - want) / len(Q)) + 0.01, (got, want)


def test_ads_estimate_is_unbiased_over_random_rotations():
    # over Haar rotations, (D/d) times the squared norm of the first d rotated
    # coordinates has mean ||x||^2 (each coordinate's square has mean
    # ||x||^2 / D); and its relative spread shrinks like 1/sqrt(d), which is
    # what makes eps = eps0 / sqrt(d) a fixed significance level
    rng = np.random.default_rng(3)
    D = 32
    x = rng.standard_normal(D)
    n2 = float(x @ x)
    est = {4: [], 16: []}
    for seed in range(4000):
        y = pca.haar_rotation(D, seed) @ x
        for d in est:
            est[d].append(D / d * float(y[:d] @ y[:d]))
    for d, v in est.items():
        v = np.asarray(v)
        assert abs(v.mean() / n2 - 1) < 4 * v.std() / n2 / np.sqrt(len(v)), d
    r = np.std(est[4]) / np.std(est[16])
    # for a uniformly random direction the first d squared coordinates sum
    # to Beta(d/2, (D-d)/2) times ||x||^2, so Var[(D/d) ...] = 2 (D-d) / (d (D+2)) ||x||^4
    want = np.sqrt((2 * (D - 4) / (4 * (D + 2))) / (2 * (D - 16) / (16 * (D + 2))))
    assert abs(r / want - 1) < 0.1, (r, want)


def test_ads_prunes_nothing_at_large_eps0_and_matches_pruning_off(small):
    idx = small["idx"]
    Q = small["Q"][:20]
    probes = idx.probe(idx.rotate_queries(Q), 8)
    S = search.n_steps(small["D"], 8)
    off = search.search(idx, Q, probes, 8, 10, 8, *search.disabled_tables(S))
    ads = search.search(idx, Q, probes, 8, 10, 8, None, None, estimator="ads", ads_eps0=1e9)
    assert np.array_equal(ads[0], off[0]) and np.array_equal(ads[1], off[1])
    assert ads[2][:, 1].sum() == 0
    tight = search.search(idx, Q, probes, 8, 10, 8, None, None, estimator="ads", ads_eps0=0.5)
    assert tight[2][:, 1].sum() > 0


def test_haar_rotation_is_orthogonal_and_uniform():
    D = 24
    R = pca.haar_rotation(D, 1)
    assert np.abs(R @ R.T - np.eye(D)).max() < 1e-12
    # the first row is uniform on the sphere: over seeds its entries have
    # mean 0 and variance 1/D, and the sign of R's determinant is +-1 at random
    rows = np.stack([pca.haar_rotation(D, s)[0] for s in range(3000)])
    assert abs(rows.mean()) < 4 / np.sqrt(rows.size * D)
    assert abs(rows.var() * D - 1) < 0.05
    dets = [np.sign(np.linalg.det(pca.haar_rotation(6, s))) for s in range(400)]
    assert 0.35 < np.mean(np.asarray(dets) > 0) < 0.65
