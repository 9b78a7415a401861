"""Pins of the oracle's IVF pieces (Section II-A): k-means, assignment, probes."""
import itertools

import numpy as np

from oracle import ivf


def test_assignment_is_brute_force_argmin_with_lower_id_on_ties():
    rng = np.random.default_rng(3)
    X = rng.integers(-3, 4, size=(200, 3)).astype(np.float64)
    C = rng.integers(-3, 4, size=(7, 3)).astype(np.float64)
    C[5] = C[2]  # duplicate centroid: ties must go to id 2
    a = ivf.assign(X, C)
    for i, x in enumerate(X):
        best = None
        for j, c in enumerate(C):
            d = sum((x[k] - c[k]) ** 2 for k in range(3))
            if best is None or d < best[0]:
                best = (d, j)
        assert a[i] == best[1]
    assert not np.any(a == 5)


def test_kmeans_objective_non_increasing_and_final_assignment_is_argmin():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((1500, 6))
    C, a, objs = ivf.kmeans(X, rng.choice(1500, 12, replace=False), 10)
    assert all(o2 <= o1 + 1e-12 for o1, o2 in zip(objs, objs[1:]))
    assert np.array_equal(a, ivf.assign(X, C))


def test_kmeans_recovers_separated_blob_means():
    rng = np.random.default_rng(9)
    centers = np.array([[0, 0], [100, 0], [0, 100], [100, 100]], dtype=np.float64)
    X = np.concatenate([c + rng.standard_normal((50, 2)) for c in centers])
    init = np.array([0, 50, 100, 150])  # one row from each blob
    C, a, _ = ivf.kmeans(X, init, 5)
    for k in range(4):
        assert np.allclose(C[k], X[50 * k:50 * (k + 1)].mean(0), atol=1e-12)
        assert np.all(a[50 * k:50 * (k + 1)] == k)


def test_probe_orders_by_distance_then_list_id():
    C = np.array([[1.0, 0], [0, 1.0], [-1.0, 0], [3.0, 0], [0, -1.0]])
    Q = np.zeros((1, 2))
    lists, d = ivf.probe(Q, C, 5)
    assert list(lists[0]) == [0, 1, 2, 4, 3]
    assert list(d[0]) == [1, 1, 1, 1, 9]


def test_lists_from_assignment_storage_order():
    a = np.array([2, 0, 2, 1, 0, 2])
    off, mem = ivf.lists_from_assignment(a, 4)
    assert list(off) == [0, 2, 3, 6, 6]
    assert list(mem) == [1, 4, 3, 0, 2, 5]
    for l, lo, hi in zip(range(4), off, off[1:]):
        assert all(a[m] == l for m in mem[lo:hi])
    assert sorted(itertools.chain(mem)) == list(range(6))
