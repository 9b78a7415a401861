"""Estimate quality on the device (Section VII, Exp-7; Section IV-B Fig. 1;
Section IV-C Fig. 2), from the partial distances the CUDA path computes over
its stored slabs (dade_partials_collect), on a whole reduced database of the
SIFT- and GIST-shaped sets (20,000 vectors, 30 queries, every bucket probed).

* recall@100 of the 32-dimension estimate against the exact top-100, for the
  PCA rotation with FP32 / BF16 / FP8 slabs and a Haar-random rotation (the
  random projection of ADS; its D/d scale does not change the ranking),
  next to the oracle's numbers for the same data (tests of the oracle in
  test_estimator_accuracy): within 0.02.
* Fig. 1: the error term <q_r, x_r> of the residual dims is more
  concentrated under PCA than under the random rotation, and shrinks as the
  projected dims grow.
* Fig. 2: the RES estimate's error dis - (p_d + ||x_r||^2 + ||q_r||^2),
  divided by the per-query sigma = 2 sqrt(sum_{i>d} q_i^2 lambda_i), has its
  99.7th percentile of |z| near 3 (the Gaussian rule), far below ADS's 10.

The histograms and quantiles are printed as one JSON line
(ESTIMATOR_FIGURES) and written to the file DADE_FIG_JSON names, if set.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import pca

from .test_estimator_accuracy import D_EST, _recall_table

pytestmark = pytest.mark.gpu

N, NQ, NLIST = 20000, 30, 16


@pytest.fixture(scope="module")
def G():
    from paper_2404_16322_gb300 import build
    build.build()
    import paper_2404_16322_gb300 as G
    return G


def _device_partials(G, X, Q, mu, R, dtype):
    idx = G.ivf_build(X, mu, R, NLIST, kmeans_iters=3, seed=1, dtype=dtype)
    try:
        out = G.dade_partials_collect(idx, Q, NLIST, 32)
    finally:
        idx.close()
    n = len(X)
    assert len(out["id"]) == len(Q) * n  # every vector, once per query
    P = out["partials"].reshape(len(Q), n, -1)
    ids = out["id"].reshape(len(Q), n)
    assert np.all(ids == np.arange(n)[None, :])  # sorted by (query, id)
    return P.astype(np.float64)


def _recall(P, exact, d_col=0):
    rec = []
    for b in range(P.shape[0]):
        top = set(np.argsort(exact[b], kind="stable")[:100].tolist())
        est = np.argsort(P[b, :, d_col], kind="stable")[:100]
        rec.append(len(top & set(est.tolist())) / 100)
    return float(np.mean(rec))


@pytest.mark.parametrize("name", ["sift1m", "gist1m"])
def test_device_estimate_recall_and_error_figures(G, name):
    spec = synth.WORKLOADS[name]["spec"]
    X = spec.sample(N, 1)
    Q = spec.sample(NQ, 2)
    D = X.shape[1]
    mu, R, lam = pca.train_rotation(X)
    Rh = pca.haar_rotation(D, 4)
    x64, q64 = X.astype(np.float64), Q.astype(np.float64)
    exact = (q64 * q64).sum(1)[:, None] + (x64 * x64).sum(1)[None, :] - 2.0 * q64 @ x64.T
    P = {k: _device_partials(G, X, Q, mu, rot, dt)
         for k, rot, dt in (("pca", R, "f32"), ("rand", Rh, "f32"), ("pca_bf16", R, "bf16"), ("pca_fp8", R, "fp8"))}
    col = D_EST // 32 - 1
    dev = {k: _recall(v, exact, col) for k, v in P.items()}
    ora = _recall_table(name)
    for k in dev:
        assert abs(dev[k] - ora[k]) <= 0.02, (k, dev[k], ora[k])

    # Fig. 1: the residual inner product <q_r, x_r> = (||q_r||^2 + ||x_r||^2 -
    # (dis - p_d)) / 2 under both rotations, from the device's p_d
    def cross(Pk, rot, d):
        Xr, Qr = pca.rotate(X, mu, rot), pca.rotate(Q, mu, rot)
        xr = (Xr[:, d:] ** 2).sum(1)
        qr = (Qr[:, d:] ** 2).sum(1)
        return 0.5 * (qr[:, None] + xr[None, :] - (exact - Pk[:, :, d // 32 - 1])), Qr

    c_pca, Qr = cross(P["pca"], R, D_EST)
    c_rand, _ = cross(P["rand"], Rh, D_EST)
    lim = 4.0 * c_rand.std()
    edges = np.linspace(-lim, lim, 41)
    fig1 = {"dims": D_EST, "residual_dims": D - D_EST, "edges": edges.tolist(),
            "pca": np.histogram(c_pca, edges)[0].tolist(), "random": np.histogram(c_rand, edges)[0].tolist(),
            "std_pca": float(c_pca.std()), "std_random": float(c_rand.std())}
    assert fig1["std_pca"] < fig1["std_random"]
    dims = [d for d in (32, 64, 96, 128) if d < D]
    stds = [float(cross(P["pca"], R, d)[0].std()) for d in dims]
    fig1["std_pca_by_dims"] = dict(zip(map(str, dims), stds))
    assert all(a > b for a, b in zip(stds, stds[1:]))

    # Fig. 2: z = error / sigma_q of the RES estimate (Eq. 1)
    fig2 = {}
    for d in (32, 128 if D > 128 else 64):
        c, Qr = cross(P["pca"], R, d)
        sigma = 2.0 * np.sqrt(((Qr[:, d:] ** 2) * lam[None, d:]).sum(1))
        z = (-2.0 * c) / sigma[:, None]
        az = np.abs(z)
        zedges = np.linspace(-6, 6, 49)
        fig2[str(d)] = {"p99.7_abs_z": float(np.percentile(az, 99.7)), "frac_above_3": float((az > 3).mean()),
                        "frac_above_10": float((az > 10).mean()), "edges": zedges.tolist(),
                        "counts": np.histogram(z, zedges)[0].tolist()}
        assert 2.0 < fig2[str(d)]["p99.7_abs_z"] < 4.5
        assert fig2[str(d)]["frac_above_10"] < 1e-4
    out = {"workload": name, "n": N, "queries": NQ, "recall@100": {"device": dev, "oracle": ora},
           "fig1": fig1, "fig2": fig2}
    print("ESTIMATOR_FIGURES", json.dumps(out))
    path = os.environ.get("DADE_FIG_JSON")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(out) + "\n")
