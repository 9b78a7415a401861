"""GPU parity of the Gaussian-bound (RES) test of Section IV-C (Algorithms
1-2, Eq. 1-2) against the oracle: pruning decisions, work accounting and
results, for FP32 and BF16 slabs, step widths, the final test, save/load
and sharding.

Both sides see the oracle's pre-rotated FP32 vectors (R = I), so the
per-dimension variances agree to FP32 rounding.  The device evaluates the
test as FP32 sums of a partial distance, a residual norm and a per-query
term whose magnitudes reach ||x||^2 + ||q||^2 (several times tau), so the
band in which a decision counts as ambiguous is the FP32-rotation one
(3e-5 tau) rather than the pre-rotated learned one."""
import numpy as np
import pytest

import synth
from oracle import search

from . import gpu_helpers as H
from . import parity

pytestmark = pytest.mark.gpu

AMB_RES = H.AMB["f32"]


@pytest.fixture(scope="module")
def G():
    from paper_2404_16322_gb300 import build
    build.build()
    import paper_2404_16322_gb300 as G
    return G


def _setup(G, dtype="f32", delta_d=16):
    X, Q, T, cfg = synth.workload("tiny", n_train=600)
    inp = H.oracle_inputs(X, T, cfg["nlist"], K=10, nprobe=8, delta_d=delta_d, dtype=dtype, n_train=600,
                          prerotate=True)
    idx = H.build_gpu(G, None, inp, cfg["nlist"], dtype=dtype, delta_d=delta_d)
    return dict(inp=inp, idx=idx, Q=inp["rot"](Q), X=inp["X"], cfg=cfg)


@pytest.fixture(scope="module")
def pre(G):
    s = _setup(G)
    yield s
    s["idx"].close()


def _oracle_res(s, K, nprobe, delta_d, m, first_wave=1, growth=1, final_rel=np.inf):
    oidx = s["inp"]["oidx"]
    P = int(np.max(nprobe))
    pr = oidx.probe(oidx.rotate_queries(s["Q"]), P)
    ids, d, st, ad = search.search(oidx, s["Q"], pr, nprobe, K, delta_d, None, None, first_wave=first_wave,
                                   growth=growth, amb=AMB_RES, final_rel=final_rel, estimator="res", res_m=m,
                                   with_amb=True)
    return ids, d, (st, ad), pr


def _check(s, out, ids, d, st, K=10):
    st, ad = st
    assert out["status"] == 0
    parity.check(out["ids"], out["dists"], ids, d, s["X"], s["Q"], K, amb_d=ad)
    un = st[:, 4] == 0
    assert np.array_equal(out["stats"][:, 0], st[:, 0])
    assert np.array_equal(out["stats"][un], st[un, :4])


@pytest.mark.parametrize("m", [0.5, 2.0, 8.0])
def test_res_matches_oracle(G, pre, m):
    ids, d, st, pr = _oracle_res(pre, 10, 8, 16, m)
    out = H.gpu_search(G, pre["idx"], pre["Q"], 10, 8, 16, probe_in=pr, estimator="res", res_m=m,
                       want=("stats",))
    _check(pre, out, ids, d, st)
    if m <= 2.0:
        assert st[0][:, 1].sum() > 0  # the test does prune at these multipliers


def test_res_smaller_multiplier_prunes_more(G, pre):
    pr = pre["inp"]["oidx"].probe(pre["Q"], 8)
    n = {}
    for m in (0.0, 1.0, 8.0, 64.0):
        out = H.gpu_search(G, pre["idx"], pre["Q"], 10, 8, 16, probe_in=pr, estimator="res", res_m=m,
                           want=("stats",))
        assert out["status"] == 0
        n[m] = out["stats"][:, 1].sum()
    assert n[0.0] >= n[1.0] >= n[8.0] >= n[64.0]
    assert n[0.0] > n[8.0]


@pytest.mark.parametrize("fw,g,final", [(2, 1, False), (2, 30, False), (2, 1, True)])
def test_res_wave_schedules_and_final_test(G, pre, fw, g, final):
    fr = search.FINAL_REL if final else np.inf
    ids, d, st, pr = _oracle_res(pre, 10, 8, 16, 1.0, first_wave=fw, growth=g, final_rel=fr)
    out = H.gpu_search(G, pre["idx"], pre["Q"], 10, 8, 16, probe_in=pr, first_wave=fw, growth=g,
                       final_test=final, estimator="res", res_m=1.0, want=("stats",))
    _check(pre, out, ids, d, st)


def test_res_ragged_K_and_nprobe(G, pre):
    rng = np.random.default_rng(11)
    B = len(pre["Q"])
    K = rng.integers(1, 21, B).astype(np.int32)
    npb = rng.integers(1, 17, B).astype(np.int32)
    ids, d, st, pr = _oracle_res(pre, K, npb, 16, 2.0)
    out = H.gpu_search(G, pre["idx"], pre["Q"], K, npb, 16, probe_in=pr, max_K=20, max_nprobe=16,
                       estimator="res", res_m=2.0)
    parity.check(out["ids"], out["dists"], ids, d, pre["X"], pre["Q"], K, amb_d=st[1])


@pytest.mark.parametrize("dtype,delta_d", [("f32", 8), ("f32", 32), ("bf16", 8), ("bf16", 16), ("fp8", 16)])
def test_res_slab_precisions_and_step_widths(G, dtype, delta_d):
    s = _setup(G, dtype, delta_d)
    try:
        amb_band = {"f32": AMB_RES, "bf16": AMB_RES, "fp8": AMB_RES}[dtype]
        oidx = s["inp"]["oidx"]
        pr = oidx.probe(oidx.rotate_queries(s["Q"]), 8)
        ids, d, st, ad = search.search(oidx, s["Q"], pr, 8, 10, delta_d, None, None, amb=amb_band,
                                       estimator="res", res_m=1.0, with_amb=True)
        out = H.gpu_search(G, s["idx"], s["Q"], 10, 8, delta_d, probe_in=pr, estimator="res", res_m=1.0,
                           want=("stats",))
        _check(s, out, ids, d, (st, ad))
    finally:
        s["idx"].close()


def test_res_needs_no_table(G, pre):
    # delta_d = 8 has no table installed on this index: the learned test is
    # refused, the RES test runs
    with pytest.raises(Exception):
        H.gpu_search(G, pre["idx"], pre["Q"][:4], 10, 8, 8)
    ids, d, st, pr = _oracle_res(pre, 10, 8, 8, 2.0)
    out = H.gpu_search(G, pre["idx"], pre["Q"], 10, 8, 8, probe_in=pr, estimator="res", res_m=2.0,
                       want=("stats",))
    _check(pre, out, ids, d, st)


def test_res_host_errors(G, pre):
    for kw in (dict(estimator="res", res_m=-1.0), dict(estimator="res", res_m=float("inf")),
               dict(estimator="res", res_m=float("nan"))):
        with pytest.raises(Exception):
            H.gpu_search(G, pre["idx"], pre["Q"][:4], 10, 8, 16, **kw)


def test_res_after_save_load(G, pre, tmp_path):
    p = str(tmp_path / "res.dade")
    G.dade_index_save(pre["idx"], p)
    idx2 = G.dade_index_load(p)
    try:
        pr = pre["inp"]["oidx"].probe(pre["Q"], 8)
        a = H.gpu_search(G, pre["idx"], pre["Q"], 10, 8, 16, probe_in=pr, estimator="res", res_m=1.0,
                         want=("stats",))
        b = H.gpu_search(G, idx2, pre["Q"], 10, 8, 16, probe_in=pr, estimator="res", res_m=1.0,
                         want=("stats",))
        assert np.array_equal(a["ids"], b["ids"]) and np.array_equal(a["dists"], b["dists"])
        assert np.array_equal(a["stats"], b["stats"])
    finally:
        idx2.close()
