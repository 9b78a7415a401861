"""Pin of the oracle's exact KNN (Section II-A) against a pure-Python loop."""
import numpy as np

from oracle import knn


def test_exact_knn_matches_python_loop_with_ties_by_id():
    rng = np.random.default_rng(4)
    X = rng.integers(0, 4, size=(60, 3)).astype(np.float32)  # many exact ties
    Q = rng.integers(0, 4, size=(7, 3)).astype(np.float32)
    ids, d = knn.exact_knn(X, Q, 9)
    for b in range(len(Q)):
        full = sorted((sum((float(X[i][k]) - float(Q[b][k])) ** 2 for k in range(3)), i)
                      for i in range(len(X)))[:9]
        assert [i for _, i in full] == list(ids[b])
        assert [dd for dd, _ in full] == list(d[b])
