"""GPU parity of OPQ-L (Section V-B "Approximate Distances": OPQ's
asymmetric distance, one three-feature learned test, then the exact
distance) against the oracle.  Both sides get the oracle's pre-rotated FP32
vectors (R = I), its dimension allocation and codebooks; the library
encodes the stored vectors itself, and the codes are compared first."""
import numpy as np
import pytest

import synth
from oracle import fit, pq, search

from . import gpu_helpers as H
from . import parity

pytestmark = pytest.mark.gpu

M = 32


@pytest.fixture(scope="module")
def G():
    from paper_2404_16322_gb300 import build
    build.build()
    import paper_2404_16322_gb300 as G
    return G


@pytest.fixture(scope="module")
def pre(G):
    X, Q, T, cfg = synth.workload("tiny", n_train=600)
    inp = H.oracle_inputs(X, T, cfg["nlist"], K=10, nprobe=8, delta_d=16, n_train=600, prerotate=True)
    idx = H.build_gpu(G, None, inp, cfg["nlist"])
    oidx = inp["oidx"]
    perm = pq.eigen_allocation(oidx.var, M)
    cb = pq.train_codebooks(oidx.Xs, perm, M, 6, np.random.default_rng(3).choice(oidx.N, pq.KSUB, replace=False))
    cb32 = cb.astype(np.float32)
    codes = pq.encode(oidx.Xs, perm, cb32.astype(np.float64))
    err = pq.quantisation_error(oidx.Xs, codes, perm, cb32.astype(np.float64))
    G.dade_pq_set(idx, perm, cb32)
    yield dict(idx=idx, inp=inp, oidx=oidx, perm=perm, cb=cb32.astype(np.float64), codes=codes, err=err,
               X=inp["X"], Q=inp["rot"](Q), T=inp["rot"](T))
    idx.close()


def test_library_allocation_equals_the_oracle(G, pre):
    perm, _ = G.dade_pq_train(pre["idx"], pre["X"][:2000], M, iters=1, seed=1)
    assert np.array_equal(perm, pq.eigen_allocation(pre["oidx"].var, M))
    G.dade_pq_set(pre["idx"], pre["perm"], pre["cb"].astype(np.float32))   # restore the oracle's quantiser


def test_codes_and_errors_match_the_oracle(G, pre):
    m, _, codes, err = G.dade_pq_get(pre["idx"], codes=True)
    assert m == M
    same = codes == pre["codes"]
    assert same.mean() > 0.9995
    # a differing code is a near tie of two centroid distances
    for r, j in zip(*np.nonzero(~same)):
        ds = pre["cb"].shape[2]
        x = pre["oidx"].Xs[r, pre["perm"][j * ds:(j + 1) * ds]]
        d = ((pre["cb"][j] - x) ** 2).sum(1)
        assert abs(d[codes[r, j]] - d[pre["codes"][r, j]]) <= 1e-5 * (1 + d.min())
    assert np.allclose(err, pre["err"], rtol=1e-4, atol=1e-5)


def _oracle_pq(s, Q, pr, nprobe, K, m1, m3, beta, mode="waves", tau=None, first_wave=1, uncertain_rows=None):
    T = pq.lut(s["oidx"].rotate_queries(Q), s["perm"], s["cb"])
    return search.search(s["oidx"], Q, pr, nprobe, K, 16, None, None, mode=mode, tau=tau, first_wave=first_wave,
                         amb=H.AMB["f32"], estimator="pq", with_amb=True, uncertain_rows=uncertain_rows,
                         pq=dict(codes=s["codes"], err=s["err"], lut=T, m1=m1, m3=m3, beta=beta))


def _code_ties(G, s):
    """Rows whose library code differs from the oracle's: they lie at near
    ties of two centroid distances (checked by test_codes_and_errors_match_
    the_oracle), so the oracle counts every decision on them as uncertain."""
    _, _, codes, _ = G.dade_pq_get(s["idx"], codes=True)
    return (codes != s["codes"]).any(1)


@pytest.mark.parametrize("coef", [(1.0, -2.0, 0.0), (0.8, -0.5, 50.0)])
def test_pq_search_matches_oracle(G, pre, coef):
    s = pre
    m1, m3, beta = coef
    G.dade_pq_set_correction(s["idx"], m1, m3, beta)
    pr = s["oidx"].probe(s["Q"], 8)
    ids, d, st, ad = _oracle_pq(s, s["Q"], pr, 8, 10, m1, m3, beta, first_wave=2, uncertain_rows=_code_ties(G, s))
    out = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, probe_in=pr, first_wave=2, estimator="pq", want=("stats",))
    assert out["status"] == 0
    parity.check(out["ids"], out["dists"], ids, d, s["X"], s["Q"], 10, amb_d=ad)
    un = st[:, 4] == 0
    assert np.array_equal(out["stats"][:, 0], st[:, 0])
    assert np.array_equal(out["stats"][un], st[un, :4])
    assert st[:, 1].sum() > 0


def test_pq_frozen_tau_and_disabled_classifier(G, pre):
    s = pre
    pr = s["oidx"].probe(s["Q"], 8)
    G.dade_pq_set_correction(s["idx"], 0.0, 0.0, -np.inf)
    off = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, probe_in=pr, estimator="pq", want=("stats",))
    full = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 0, mode="full", probe_in=pr)
    assert np.array_equal(off["ids"], full["ids"]) and np.array_equal(off["dists"], full["dists"])
    assert off["stats"][:, 1].sum() == 0
    # tau just above the 10th distance, so that no distance lies within FP32
    # rounding of it
    tau = (full["dists"][:, 9].astype(np.float64) * (1 + 1e-4)).astype(np.float32)
    G.dade_pq_set_correction(s["idx"], 1.0, -2.0, 0.0)
    ids, d, st, ad = _oracle_pq(s, s["Q"], pr, 8, 10, 1.0, -2.0, 0.0, mode="frozen", tau=tau.astype(np.float64),
                                uncertain_rows=_code_ties(G, s))
    out = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, probe_in=pr, tau=tau, estimator="pq", want=("stats",))
    assert out["status"] == 0
    parity.check(out["ids"], out["dists"], ids, d, s["X"], s["Q"], 10, amb_d=ad)


def test_pq_fit_end_to_end_keeps_recall(G, pre):
    s = pre
    m1, m3, beta = G.dade_pq_fit_correction(s["idx"], s["T"][:500], 10, 8, target_recall=0.995, seed=2)
    assert np.isfinite(beta) and m1 > 0
    pr = s["oidx"].probe(s["Q"], 8)
    out = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, probe_in=pr, estimator="pq", want=("stats",))
    full = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 0, mode="full", probe_in=pr)
    assert out["status"] == 0
    rec = parity.recall(out["ids"], full["ids"], 10)
    assert rec >= 0.97
    assert out["stats"][:, 1].sum() > 0.3 * out["stats"][:, 0].sum()
    for b in range(len(s["Q"])):
        v = out["ids"][b] >= 0
        ex = ((s["X"][out["ids"][b][v]].astype(np.float64) - s["Q"][b].astype(np.float64)) ** 2).sum(1)
        assert np.allclose(out["dists"][b][v], ex, rtol=1e-5)


def test_pq_host_errors(G, pre):
    from paper_2404_16322_gb300 import _lib
    with pytest.raises(_lib.DadeError):
        G.dade_pq_set(pre["idx"], np.zeros(pre["X"].shape[1], np.int32), pre["cb"].astype(np.float32))
    with pytest.raises(_lib.DadeError):
        H.gpu_search(G, pre["idx"], pre["Q"][:4], 10, 8, 16, estimator="pq", final_test=True)


def test_pq_survives_save_and_load(G, pre, tmp_path):
    s = pre
    G.dade_pq_set_correction(s["idx"], 1.0, -2.0, 0.0)
    p = str(tmp_path / "pq.dade")
    G.dade_index_save(s["idx"], p)
    idx2 = G.dade_index_load(p)
    try:
        m, c3, codes, err = G.dade_pq_get(idx2, codes=True)
        _, c3a, codes_a, err_a = G.dade_pq_get(s["idx"], codes=True)
        assert m == M and c3 == c3a
        assert np.array_equal(codes, codes_a) and np.array_equal(err, err_a)
        pr = s["oidx"].probe(s["Q"], 8)
        a = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, probe_in=pr, estimator="pq", want=("stats",))
        b = H.gpu_search(G, idx2, s["Q"], 10, 8, 16, probe_in=pr, estimator="pq", want=("stats",))
        assert np.array_equal(a["ids"], b["ids"]) and np.array_equal(a["stats"], b["stats"])
    finally:
        idx2.close()
