"""GPU parity of the ADS baseline (Section III: a Haar-random rotation and
the test (D/d) dis'_s > (1 + eps0/sqrt(d)) tau) run by the search kernels
through the table from dade_ads_table, against the oracle's own ADS test.

The oracle's Haar rotation is applied up front (both sides see the same
FP32 rotated vectors, R = I), so decisions differ only inside the FP32
rounding band of the test."""
import numpy as np
import pytest

import synth
from oracle import ivf, knn, pca, search

from . import gpu_helpers as H
from . import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2404_16322_gb300 import build
    build.build()
    import paper_2404_16322_gb300 as G
    return G


@pytest.fixture(scope="module")
def haar(G):
    X, Q, T, cfg = synth.workload("tiny")
    D = X.shape[1]
    mu = X.astype(np.float64).mean(0)
    Rh = pca.haar_rotation(D, 17)
    Xr = pca.rotate(X, mu, Rh).astype(np.float32)
    Qr = pca.rotate(Q, mu, Rh).astype(np.float32)
    init = np.random.default_rng(7).choice(len(Xr), cfg["nlist"], replace=False)
    C, a, _ = ivf.kmeans(Xr.astype(np.float64), init, 8)
    C32 = C.astype(np.float32)
    oidx = search.OracleIndex(Xr, np.zeros(D), np.eye(D), C32.astype(np.float64), a)
    idx = G.ivf_build(Xr, np.zeros(D), np.eye(D), cfg["nlist"], centroids=C32, assign=a)
    yield dict(X=Xr, Q=Qr, oidx=oidx, idx=idx, D=D, X0=X, Q0=Q, mu=mu, Rh=Rh, cfg=cfg, C32=C32, a=a)
    idx.close()


@pytest.mark.parametrize("delta_d,eps0", [(32, 2.1), (16, 2.1), (8, 1.0)])
def test_ads_matches_oracle(G, haar, delta_d, eps0):
    s = haar
    m1, beta = G.dade_ads_table(s["D"], delta_d, eps0)
    G.dade_set_correction(s["idx"], delta_d, m1, beta)
    pr = s["oidx"].probe(s["oidx"].rotate_queries(s["Q"]), 8)
    ids, d, st, ad = search.search(s["oidx"], s["Q"], pr, 8, 10, delta_d, None, None, estimator="ads",
                                   ads_eps0=eps0, amb=H.AMB["exact"], with_amb=True, norm_eps=H.NORM_EPS)
    out = H.gpu_search(G, s["idx"], s["Q"], 10, 8, delta_d, probe_in=pr, want=("stats",))
    assert out["status"] == 0
    parity.check(out["ids"], out["dists"], ids, d, s["X"], s["Q"], 10, amb_d=ad)
    un = st[:, 4] == 0
    assert np.array_equal(out["stats"][:, 0], st[:, 0])
    assert np.array_equal(out["stats"][un], st[un, :4])
    assert st[:, 1].sum() > 0


def test_ads_with_the_device_rotating(G, haar):
    # the library's own Haar rotation applied by ivf_build: results are valid
    # top-K lists of exact distances with recall close to pruning off
    s = haar
    D = s["D"]
    Rl = G.dade_random_rotation(D, seed=3)
    idx = G.ivf_build(s["X0"], s["mu"], Rl, s["cfg"]["nlist"], kmeans_iters=6, seed=2)
    try:
        m1, beta = G.dade_ads_table(D, 32, 2.1)
        G.dade_set_correction(idx, 32, m1, beta)
        out = H.gpu_search(G, idx, s["Q0"], 10, 16, 32, want=("stats",))
        full = H.gpu_search(G, idx, s["Q0"], 10, 16, 0, mode="full")
        assert out["status"] == 0
        X0, Q0 = s["X0"], s["Q0"]
        for b in range(len(Q0)):
            v = out["ids"][b] >= 0
            ex = ((X0[out["ids"][b][v]].astype(np.float64) - Q0[b].astype(np.float64)) ** 2).sum(1)
            assert np.allclose(out["dists"][b][v], ex, rtol=1e-5)
        gi, _ = knn.exact_knn(X0, Q0, 10)
        assert parity.recall(out["ids"], gi, 10) >= parity.recall(full["ids"], gi, 10) - 0.03
        assert out["stats"][:, 1].sum() > 0
    finally:
        idx.close()
