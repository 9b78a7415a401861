"""GPU parity: the CUDA path against the oracle on the same seeded inputs.

Both sides get the oracle's rotation, centroids, bucket assignment and
correction tables; the comparisons follow tests/parity.py."""
import numpy as np
import pytest

import synth
from oracle import ivf, knn, search

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
def tiny_setup(G):
    """The small workload with the rotation done by each side (FP64 oracle,
    FP32 GEMM on the device)."""
    X, Q, T, cfg = synth.workload("tiny")
    inp = H.oracle_inputs(X, T, cfg["nlist"], K=10, nprobe=8, delta_d=16)
    idx = H.build_gpu(G, X, inp, cfg["nlist"])
    return dict(X=X, Q=Q, T=T, cfg=cfg, inp=inp, idx=idx, amb="f32")


@pytest.fixture(scope="module")
def tiny_pre(G):
    """The small workload pre-rotated by the oracle: both sides see the same
    FP32 rotated vectors (R = I), so only FP32 accumulation differs."""
    X, Q, T, cfg = synth.workload("tiny")
    inp = H.oracle_inputs(X, T, cfg["nlist"], K=10, nprobe=8, delta_d=16, prerotate=True)
    idx = H.build_gpu(G, None, inp, cfg["nlist"])
    return dict(X=inp["X"], Q=inp["rot"](Q), cfg=cfg, inp=inp, idx=idx, amb="exact")


def _oracle(s, Q, K, nprobe, delta_d=16, m1=None, beta=None, mode="waves", tau=None, dtype_amb=None,
            oidx=None, probes=None):
    dtype_amb = dtype_amb or s.get("amb", "f32")
    oidx = oidx or s["inp"]["oidx"]
    P = int(np.max(nprobe))
    pr = probes if probes is not None else oidx.probe(oidx.rotate_queries(Q), P)
    m1 = s["inp"]["m1"] if m1 is None else m1
    beta = s["inp"]["beta"] if beta is None else beta
    ids, d, st, ad = search.search(oidx, Q, pr, nprobe, K, delta_d, m1.astype(np.float64),
                                   beta.astype(np.float64), mode=mode, tau=tau, amb=H.AMB[dtype_amb], with_amb=True, norm_eps=H.NORM_EPS,
                                   qdev_eps=s["inp"]["qdev"])
    return ids, d, st, pr, ad


def test_rotated_queries_match_oracle(G, tiny_setup):
    s = tiny_setup
    out = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, want=("qrot",))
    ref = s["inp"]["oidx"].rotate_queries(s["Q"])
    err = np.abs(out["qrot"] - ref).max(axis=1) / np.linalg.norm(ref, axis=1)
    # the oracle's rounding model assumes at most FLIP_EPS (the same GEMM
    # rotates the database)
    assert err.max() < H.FLIP_EPS


def test_probes_match_oracle_up_to_near_ties(G, tiny_setup):
    s = tiny_setup
    P = 8
    out = H.gpu_search(G, s["idx"], s["Q"], 10, P, 16, want=("probes",))
    oidx = s["inp"]["oidx"]
    Qr = oidx.rotate_queries(s["Q"])
    d = ivf.sq_dists(Qr, oidx.C)
    lists, _ = ivf.probe(Qr, oidx.C, oidx.nlist)
    n_exact = 0
    for b in range(len(s["Q"])):
        g, o = out["probes"][b], lists[b, :P]
        if np.array_equal(g, o):
            n_exact += 1
            continue
        # a difference is allowed only among centroids within 1e-5 of the boundary
        kth = d[b, lists[b, P - 1]]
        for l in set(g) ^ set(o):
            assert abs(d[b, l] - kth) <= 1e-5 * kth
    assert n_exact >= 0.95 * len(s["Q"])


@pytest.mark.parametrize("kernel", ["tensor", "cuda"])
@pytest.mark.parametrize("setup", ["tiny_setup", "tiny_pre"])
@pytest.mark.parametrize("mode", ["waves", "tables_off"])
def test_prune_path_matches_oracle(G, request, setup, mode, kernel):
    s = request.getfixturevalue(setup)
    Q = s["Q"]
    if mode == "waves":
        ids, d, st, pr, ad = _oracle(s, Q, 10, 8)
        out = H.gpu_search(G, s["idx"], Q, 10, 8, 16, probe_in=pr, want=("stats",), scan_kernel=kernel)
    else:
        S = search.n_steps(128, 16)
        m1, beta = search.disabled_tables(S)
        ids, d, st, pr, ad = _oracle(s, Q, 10, 8, m1=m1, beta=beta)
        G.dade_set_correction(s["idx"], 16, m1.astype(np.float32), beta.astype(np.float32))
        try:
            out = H.gpu_search(G, s["idx"], Q, 10, 8, 16, probe_in=pr, want=("stats",), scan_kernel=kernel)
        finally:
            G.dade_set_correction(s["idx"], 16, s["inp"]["m1"], s["inp"]["beta"])
    assert out["status"] == 0
    parity.check(out["ids"], out["dists"], ids, d, s["X"], Q, 10, amb_d=ad)
    # work accounting equals the oracle's wherever no decision was ambiguous
    un = st[:, 4] == 0
    assert np.array_equal(out["stats"][:, 0], st[:, 0])
    assert np.array_equal(out["stats"][un], st[un, :4])
    assert st[:, 1].sum() > 0 or mode != "waves"


def test_full_scan_matches_oracle_exact_over_probed(G, tiny_setup):
    s = tiny_setup
    S = search.n_steps(128, 16)
    ids, d, st, pr, ad = _oracle(s, s["Q"], 10, 8, m1=search.disabled_tables(S)[0],
                             beta=search.disabled_tables(S)[1])
    out = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 0, mode="full", probe_in=pr)
    parity.check(out["ids"], out["dists"], ids, d, s["X"], s["Q"], 10, amb_d=None)


def test_end_to_end_without_given_probes(G, tiny_setup):
    s = tiny_setup
    out = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, want=("probes",))
    ids, d, st, pr, ad = _oracle(s, s["Q"], 10, 8)
    # the device's own probes differ from the FP64 ones only at near-ties of
    # centroid distances; queries whose probe lists differ are compared with
    # the oracle run on the device's probe list (still every rank below amb_d)
    same = np.all(out["probes"] == pr, axis=1)
    assert same.mean() >= 0.95
    if not same.all():
        i2, d2, _, _, a2 = _oracle(s, s["Q"], 10, 8, probes=out["probes"])
        ids, d, ad = ids.copy(), d.copy(), ad.copy()
        ids[~same], d[~same], ad[~same] = i2[~same], d2[~same], a2[~same]
    parity.check(out["ids"], out["dists"], ids, d, s["X"], s["Q"], 10, amb_d=ad)


def test_frozen_tau_matches_oracle(G, tiny_pre):
    s = tiny_pre
    S = search.n_steps(128, 16)
    _, d0, _, pr, ad = _oracle(s, s["Q"], 10, 8, m1=search.disabled_tables(S)[0],
                           beta=search.disabled_tables(S)[1])
    tau = (d0[:, -1] * 1.05).astype(np.float32)
    ids, d, st, _, ad = _oracle(s, s["Q"], 10, 8, mode="frozen", tau=tau.astype(np.float64), probes=pr)
    out = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, probe_in=pr, tau=tau)
    parity.check(out["ids"], out["dists"], ids, d, s["X"], s["Q"], 10, amb_d=ad)


@pytest.mark.parametrize("fw,g", [(2, 2), (2, 30)])
def test_wave_growth_schedules(G, tiny_pre, fw, g):
    """Waves [0,f), [f, f*2^g), ...: the oracle's waves mode with the same
    schedule gives the same ids (strict up to the ambiguity band)."""
    s = tiny_pre
    oidx = s["inp"]["oidx"]
    pr = oidx.probe(oidx.rotate_queries(s["Q"]), 8)
    ids, d, st, ad = search.search(oidx, s["Q"], pr, 8, 10, 16, s["inp"]["m1"].astype(np.float64),
                                   s["inp"]["beta"].astype(np.float64), first_wave=fw, growth=g,
                                   amb=H.AMB["exact"], with_amb=True, norm_eps=H.NORM_EPS)
    out = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, probe_in=pr, first_wave=fw, growth=g, want=("stats",))
    assert out["status"] == 0
    parity.check(out["ids"], out["dists"], ids, d, s["X"], s["Q"], 10, amb_d=ad)
    un = st[:, 4] == 0
    assert np.array_equal(out["stats"][un], st[un, :4])


def test_final_test_on_completed_distance(G, tiny_pre):
    """With the test on the completed rotated distance both sides drop the
    same candidates before the exact distance; results do not change."""
    s = tiny_pre
    oidx = s["inp"]["oidx"]
    pr = oidx.probe(oidx.rotate_queries(s["Q"]), 8)
    args = (oidx, s["Q"], pr, 8, 10, 16, s["inp"]["m1"].astype(np.float64), s["inp"]["beta"].astype(np.float64))
    ids, d, st, ad = search.search(*args, first_wave=2, amb=H.AMB["exact"], final_rel=search.FINAL_REL,
                                   with_amb=True, norm_eps=H.NORM_EPS)
    out = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, probe_in=pr, first_wave=2, final_test=True,
                       want=("stats",))
    off = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, probe_in=pr, first_wave=2, want=("stats",))
    assert out["status"] == 0
    parity.check(out["ids"], out["dists"], ids, d, s["X"], s["Q"], 10, amb_d=ad)
    un = st[:, 4] == 0
    assert np.array_equal(out["stats"][un], st[un, :4])
    assert np.array_equal(out["ids"], off["ids"]) and np.array_equal(out["dists"], off["dists"])
    assert out["stats"][:, 2].sum() < off["stats"][:, 2].sum()


def test_ragged_K_and_nprobe(G, tiny_pre):
    s = tiny_pre
    rng = np.random.default_rng(5)
    B = len(s["Q"])
    K = rng.integers(1, 21, B).astype(np.int32)
    npb = rng.integers(1, 17, B).astype(np.int32)
    ids, d, st, pr, ad = _oracle(s, s["Q"], K, npb)
    out = H.gpu_search(G, s["idx"], s["Q"], K, npb, 16, probe_in=pr, max_K=20, max_nprobe=16)
    parity.check(out["ids"], out["dists"], ids, d, s["X"], s["Q"], K, amb_d=ad)
    for b in range(B):  # beyond each query's K the output is padding
        assert np.all(out["ids"][b, K[b]:] == -1)


@pytest.mark.parametrize("kernel", ["tensor", "cuda"])
@pytest.mark.parametrize("dtype,delta_d", [("f32", 8), ("f32", 32), ("bf16", 8), ("bf16", 16),
                                           ("bf16", 32), ("fp8", 8), ("fp8", 16), ("fp8", 32)])
def test_slab_precisions_and_step_widths_strict(G, dtype, delta_d, kernel):
    # pre-rotated inputs: both sides quantise the same FP32 values
    X, Q, T, cfg = synth.workload("tiny", n_train=600)
    inp = H.oracle_inputs(X, T, cfg["nlist"], K=10, nprobe=8, delta_d=delta_d, dtype=dtype, n_train=600,
                          prerotate=True)
    idx = H.build_gpu(G, None, inp, cfg["nlist"], dtype=dtype, delta_d=delta_d)
    s = dict(inp=inp)
    Qr = inp["rot"](Q)
    ids, d, st, pr, ad = _oracle(s, Qr, 10, 8, delta_d=delta_d, dtype_amb="exact")
    out = H.gpu_search(G, idx, Qr, 10, 8, delta_d, probe_in=pr, want=("stats",), scan_kernel=kernel)
    parity.check(out["ids"], out["dists"], ids, d, inp["X"], Qr, 10, amb_d=ad)
    un = st[:, 4] == 0
    assert np.array_equal(out["stats"][un], st[un, :4])
    idx.close()


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_low_precision_slabs_with_device_rotation(G, dtype):
    # the device rotates and quantises its own FP32 values: a coordinate
    # within the rotation's rounding of a midpoint of the format may be
    # stored at the neighbouring value (and an FP8 scale may move); the
    # oracle bounds that per coordinate (Xdev), so ids are still compared at
    # every rank below amb_d, plus recall against the exact top-K
    X, Q, T, cfg = synth.workload("tiny", n_train=600)
    inp = H.oracle_inputs(X, T, cfg["nlist"], K=10, nprobe=8, delta_d=16, dtype=dtype, n_train=600)
    idx = H.build_gpu(G, X, inp, cfg["nlist"], dtype=dtype, delta_d=16)
    s = dict(inp=inp)
    ids, d, st, pr, ad = _oracle(s, Q, 10, 8, dtype_amb=dtype)
    out = H.gpu_search(G, idx, Q, 10, 8, 16, probe_in=pr)
    parity.check(out["ids"], out["dists"], ids, d, X, Q, 10, amb_d=ad)
    S = search.n_steps(128, 16)
    top, _, _, _, ad = _oracle(s, Q, 10, 8, m1=search.disabled_tables(S)[0], beta=search.disabled_tables(S)[1],
                           probes=pr)
    assert parity.recall(out["ids"], top, 10) >= parity.recall(ids, top, 10) - 0.02
    idx.close()


def test_multi_tile_buckets_many_queries_and_ragged_dimension(G):
    # D = 100 (not a multiple of 8), 6 buckets of ~1000 vectors (several
    # 256-candidate tiles), 300 queries (several 16-query groups per bucket).
    spec = synth.MixtureSpec(D=100, n_comp=6, alpha=0.9)
    X = spec.sample(6000, 1)
    Q = spec.sample(300, 2)
    T = spec.sample(400, 3)
    inp = H.oracle_inputs(X, T, 6, K=20, nprobe=3, delta_d=16, n_train=400, prerotate=True)
    idx = H.build_gpu(G, None, inp, 6)
    s = dict(inp=inp)
    X, Q = inp["X"], inp["rot"](Q)
    ids, d, st, pr, ad = _oracle(s, Q, 20, 3, dtype_amb="exact")
    out = H.gpu_search(G, idx, Q, 20, 3, 16, probe_in=pr, want=("stats",))
    parity.check(out["ids"], out["dists"], ids, d, X, Q, 20, amb_d=ad)
    assert np.array_equal(out["stats"][:, 0], st[:, 0])
    # all buckets probed with pruning off: exact KNN
    S = search.n_steps(100, 16)
    out = H.gpu_search(G, idx, Q, 20, 6, 0, mode="full")
    gi, gd = knn.exact_knn(X, Q, 20)
    parity.check(out["ids"], out["dists"], gi, gd, X, Q, 20, amb_d=None)
    del S
    idx.close()


def test_large_K_padding_and_empty_batch(G, tiny_setup):
    s = tiny_setup
    # K larger than the probed candidates: the tail pads with -1 / +inf
    ids, d, st, pr, ad = _oracle(s, s["Q"][:5], 1024, 1)
    out = H.gpu_search(G, s["idx"], s["Q"][:5], 1024, 1, 16, probe_in=pr)
    parity.check(out["ids"], out["dists"], ids, d, s["X"], s["Q"][:5], 1024, amb_d=ad)
    assert (out["ids"] == -1).any()
    out = H.gpu_search(G, s["idx"], s["Q"][:0], 10, 8, 16, max_K=10, max_nprobe=8)
    assert out["ids"].shape == (0, 10)


def test_device_status_reports_bad_per_query_values(G, tiny_setup):
    s = tiny_setup
    K = np.full(len(s["Q"]), 10, np.int32)
    K[3] = 50  # above max_K
    out = H.gpu_search(G, s["idx"], s["Q"], K, 8, 16, max_K=10)
    assert out["status"] == 1
    assert np.all(out["ids"][3] == -1)


def test_host_errors(G, tiny_setup):
    from paper_2404_16322_gb300 import _lib
    s = tiny_setup
    with pytest.raises(_lib.DadeError) as e:
        H.gpu_search(G, s["idx"], s["Q"], 10, 8, 32)  # no table for delta_d = 32
    assert e.value.status == 5
    with pytest.raises(_lib.DadeError):
        H.gpu_search(G, s["idx"], s["Q"], 10, 8, 12)
    with pytest.raises(_lib.DadeError):
        H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, max_K=2000)
    with pytest.raises(_lib.DadeError) as e:
        H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, test_steps=2, final_test=True)
    assert e.value.status == 6
    with pytest.raises(_lib.DadeError):
        H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, test_steps=-1)


def test_save_load_roundtrip(G, tiny_setup, tmp_path):
    s = tiny_setup
    p = tmp_path / "tiny.dade"
    G.dade_index_save(s["idx"], str(p))
    idx2 = G.dade_index_load(str(p))
    a = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16)
    b = H.gpu_search(G, idx2, s["Q"], 10, 8, 16)
    assert np.array_equal(a["ids"], b["ids"]) and np.array_equal(a["dists"], b["dists"])
    raw = bytearray(p.read_bytes())
    raw[len(raw) // 2] ^= 0xFF
    p.write_bytes(bytes(raw))
    from paper_2404_16322_gb300 import _lib
    with pytest.raises(_lib.DadeError):
        G.dade_index_load(str(p))
    idx2.close()


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_save_load_roundtrip_quantised_slabs(G, tmp_path, dtype):
    # the quantisation error norms travel with the file: identical results
    # and identical pruning statistics after a reload
    X, Q, T, cfg = synth.workload("tiny")
    mu, R, _ = G.dade_train_rotation(X)
    idx = G.ivf_build(X, mu, R, cfg["nlist"], kmeans_iters=4, seed=3, dtype=dtype)
    G.dade_fit_correction(idx, T[:500], 10, 8, 16)
    p = tmp_path / f"tiny_{dtype}.dade"
    G.dade_index_save(idx, str(p))
    idx2 = G.dade_index_load(str(p))
    a = H.gpu_search(G, idx, Q, 10, 8, 16, want=("stats",))
    b = H.gpu_search(G, idx2, Q, 10, 8, 16, want=("stats",))
    assert a["status"] == 0 and b["status"] == 0
    for k in ("ids", "dists", "stats"):
        assert np.array_equal(a[k], b[k]), k
    assert a["stats"][:, 1].sum() > 0
    idx2.close()
    idx.close()


def test_library_build_and_fit_end_to_end(G):
    # The library's own rotation, k-means and fitted correction: invariants
    # and recall against exact KNN.
    X, Q, T, cfg = synth.workload("tiny")
    mu, R, lam = G.dade_train_rotation(X)
    idx = G.ivf_build(X, mu, R, cfg["nlist"], kmeans_iters=8, seed=3)
    a = G.dade_index_assignment(idx)
    C = G.dade_index_centroids(idx)
    Xr = (X.astype(np.float64) - mu) @ R.T
    d = ivf.sq_dists(Xr[:2000], C.astype(np.float64))
    best = d.min(axis=1)
    assert np.all(d[np.arange(2000), a[:2000]] <= best * (1 + 1e-5) + 1e-6)
    m1, beta = G.dade_fit_correction(idx, T, 10, 8, 16)
    assert np.all(np.isfinite(m1)) and np.any(np.isfinite(beta))
    out = H.gpu_search(G, idx, Q, 10, 8, 16, want=("stats",))
    full = H.gpu_search(G, idx, Q, 10, 8, 0, mode="full")
    gi, _ = knn.exact_knn(X, Q, 10)
    r_prune = parity.recall(out["ids"], gi, 10)
    r_full = parity.recall(full["ids"], gi, 10)
    assert r_prune >= r_full - 0.02
    assert out["stats"][:, 1].sum() > 0.5 * out["stats"][:, 0].sum()
    idx.close()


@pytest.mark.parametrize("L", [1, 3])
def test_tested_steps_limit_matches_disabled_later_steps(G, tiny_pre, L):
    """test_steps = L tests only the first L steps and sends their survivors
    to the exact distance: the oracle runs the same search with every later
    step of the table disabled (m1 = 0, beta = -inf)."""
    s = tiny_pre
    m1 = s["inp"]["m1"].astype(np.float64).copy()
    beta = s["inp"]["beta"].astype(np.float64).copy()
    m1[L:], beta[L:] = 0.0, -np.inf
    ids, d, st, pr, ad = _oracle(s, s["Q"], 10, 8, m1=m1, beta=beta)
    out = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, probe_in=pr, test_steps=L, want=("stats",))
    assert out["status"] == 0
    parity.check(out["ids"], out["dists"], ids, d, s["X"], s["Q"], 10, amb_d=ad)
    un = st[:, 4] == 0
    assert np.array_equal(out["stats"][un], st[un, :4])


@pytest.mark.parametrize("kernel", ["tensor", "cuda"])
@pytest.mark.parametrize("fw,g", [(1, 1), (2, 30)])
def test_passes_within_a_wave_change_nothing(G, tiny_pre, kernel, fw, g):
    """A candidate budget below one bucket's worth makes every wave run one
    probe rank per pass, each pass tested against the wave's tau: ids,
    distances and work counters are those of one pass per wave, and agree
    with the oracle's waves."""
    s = tiny_pre
    oidx = s["inp"]["oidx"]
    pr = oidx.probe(oidx.rotate_queries(s["Q"]), 8)
    one = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, probe_in=pr, first_wave=fw, growth=g, scan_kernel=kernel,
                       want=("stats",))
    many = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, probe_in=pr, first_wave=fw, growth=g, scan_kernel=kernel,
                        want=("stats",), candidate_budget_bytes=1)
    assert one["status"] == 0 and many["status"] == 0
    for k in ("ids", "dists", "stats"):
        assert np.array_equal(one[k], many[k]), k
    oi, od, ost, oad = search.search(oidx, s["Q"], pr, 8, 10, 16, s["inp"]["m1"].astype(np.float64),
                                     s["inp"]["beta"].astype(np.float64), first_wave=fw, growth=g,
                                     amb=H.AMB["exact"], with_amb=True, norm_eps=H.NORM_EPS)
    parity.check(many["ids"], many["dists"], oi, od, s["X"], s["Q"], 10, amb_d=oad)
    small = G.dade_search_workspace_size(s["idx"], 100, 16, 10, 8, first_wave=fw, wave_growth_log2=g,
                                         candidate_budget_bytes=1)
    big = G.dade_search_workspace_size(s["idx"], 100, 16, 10, 8, first_wave=fw, wave_growth_log2=g)
    assert small <= big


@pytest.mark.parametrize("kernel,qpu", [("tensor", 16), ("tensor", 48), ("cuda", 4)])
def test_queries_per_unit_changes_nothing(G, tiny_pre, kernel, qpu):
    """Fewer queries per work unit (more units, each staging its tile for
    fewer queries): the same ids, distances and work counters."""
    s = tiny_pre
    oidx = s["inp"]["oidx"]
    pr = oidx.probe(oidx.rotate_queries(s["Q"]), 8)
    kw = dict(probe_in=pr, first_wave=2, growth=30, scan_kernel=kernel, want=("stats",))
    a = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, **kw)
    b = H.gpu_search(G, s["idx"], s["Q"], 10, 8, 16, queries_per_unit=qpu, **kw)
    assert a["status"] == 0 and b["status"] == 0
    for k in ("ids", "dists", "stats"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("nlist,B", [(400, 5), (400, 300), (400, 3000), (2000, 300), (2000, 3000)])
def test_probe_lists_at_several_batch_sizes(G, nlist, B):
    """The probe step (pipelined tensor-core centroid distances on pre-split
    operands, then the top-nprobe selection) on 400 buckets (three full
    128-centroid tiles and a ragged one: the histogram selection) and 2,000
    buckets (16 tiles: the one-pass selection under the threshold from the
    tiles' 4 smallest, with the histogram path for rows where more than 128
    scores fall below it) for 5 / 300 / 3,000 queries (a partial query
    tile): each list is the nprobe nearest by FP64 distance, sorted, up to
    centroids within 1e-5 of the boundary; per-query nprobe honoured, -1
    beyond it and for inactive slots."""
    import synth as S
    X, Q, T, cfg = S.workload("sift1m", N=60_000, n_queries=B)
    mean, R, _ = G.dade_train_rotation(X, sample_n=20_000, seed=1)
    idx = G.ivf_build(X, mean, R, nlist, kmeans_iters=3, seed=1)
    try:
        G.dade_set_correction(idx, 16, np.ones(7, np.float32), np.full(7, -np.inf, np.float32))
        rng = np.random.default_rng(B)
        npb = rng.integers(1, 65, B).astype(np.int32)
        K = np.full(B, 10, np.int32)
        if B > 5:
            K[::11] = 0
            npb[::11] = 0  # inactive slots
        out = H.gpu_search(G, idx, Q, K, npb, 16, max_nprobe=64, want=("probes", "qrot"))
        assert out["status"] == 0
        C = G.dade_index_centroids(idx).astype(np.float64)
        qr = out["qrot"].astype(np.float64)
        d = (qr * qr).sum(1)[:, None] + (C * C).sum(1)[None, :] - 2.0 * qr @ C.T
        same = 0
        for b in range(B):
            n = int(npb[b])
            f = out["probes"][b]
            assert np.all(f[n:] == -1)
            if n == 0:
                continue
            assert len(set(f[:n].tolist())) == n and np.all(f[:n] >= 0)
            assert np.all(np.diff(d[b, f[:n]]) >= -1e-5 * d[b, f[:n]].max())  # sorted by distance
            ref = np.lexsort((np.arange(len(C)), d[b]))[:n]
            if np.array_equal(f[:n], ref):
                same += 1
                continue
            kth = d[b, ref[-1]]
            for l in set(f[:n].tolist()) ^ set(ref.tolist()):
                assert abs(d[b, l] - kth) <= 1e-5 * kth
        assert same >= 0.95 * int((npb > 0).sum())
    finally:
        idx.close()


def test_probe_selection_with_massive_ties(G):
    """Twelve distinct centroids, each repeated about 170 times over 2,048
    buckets (every 128-centroid tile holds ~10 copies of each): a query's
    scores tie in blocks of ~170, more than the one-pass selection holds, so
    every row takes the histogram path.  The lists must be the nprobe
    smallest by (distance, list id): the lowest ids among the nearest
    centroid's copies."""
    X, Q, T, cfg = synth.workload("tiny", n_queries=64)
    mean, R, _ = G.dade_train_rotation(X)
    Xr = (X.astype(np.float64) - mean) @ R.T
    rng = np.random.default_rng(12)
    C12 = Xr[rng.choice(len(X), 12, replace=False)].astype(np.float32)
    nlist = 2048
    C = C12[np.arange(nlist) % 12]
    near = np.argmin(((Xr[:, None, :] - C12[None, :, :].astype(np.float64)) ** 2).sum(-1), axis=1)
    copies = (nlist - 1 - near) // 12 + 1  # copies of centroid j: ids j, j + 12, ...
    assign = (near + 12 * (np.arange(len(X)) % copies)).astype(np.int32)
    idx = G.ivf_build(X, mean, R, nlist, centroids=C, assign=assign)
    try:
        G.dade_set_correction(idx, 16, np.ones(7, np.float32), np.full(7, -np.inf, np.float32))
        P = 64
        npb = np.random.default_rng(3).integers(1, P + 1, len(Q)).astype(np.int32)
        out = H.gpu_search(G, idx, Q, 10, npb, 16, max_nprobe=P, want=("probes", "qrot"))
        assert out["status"] == 0
        Cd = G.dade_index_centroids(idx).astype(np.float64)
        qr = out["qrot"].astype(np.float64)
        d = (qr * qr).sum(1)[:, None] + (Cd * Cd).sum(1)[None, :] - 2.0 * qr @ Cd.T
        for b in range(len(Q)):
            n = int(npb[b])
            ref = np.lexsort((np.arange(nlist), d[b]))[:n]
            assert np.array_equal(out["probes"][b, :n], ref), b
            assert np.all(out["probes"][b, n:] == -1)
    finally:
        idx.close()


def test_ids_beyond_32_bits(G, tiny_pre):
    """The same index with ids 10^12 + 7 i instead of i (the merges then
    carry 64-bit ids instead of 32-bit ones): the same results through the
    id map, ties included (the map is increasing)."""
    s = tiny_pre
    inp = s["inp"]
    X = inp["X"]
    big = (10 ** 12 + 7 * np.arange(len(X))).astype(np.int64)
    a = H.build_gpu(G, None, inp, s["cfg"]["nlist"])
    b = G.ivf_build(X, inp["mu"], inp["R"], s["cfg"]["nlist"], centroids=inp["C32"], assign=inp["assign"], ids=big)
    try:
        G.dade_set_correction(b, 16, inp["m1"], inp["beta"])
        for kw in (dict(K=10, nprobe=8), dict(K=100, nprobe=16)):
            ra = H.gpu_search(G, a, s["Q"], kw["K"], kw["nprobe"], 16, first_wave=2, growth=30, want=("stats",))
            rb = H.gpu_search(G, b, s["Q"], kw["K"], kw["nprobe"], 16, first_wave=2, growth=30, want=("stats",))
            assert ra["status"] == 0 and rb["status"] == 0
            mapped = np.where(ra["ids"] >= 0, big[np.maximum(ra["ids"], 0)], -1)
            assert np.array_equal(mapped, rb["ids"])
            assert np.array_equal(ra["dists"], rb["dists"])
            assert np.array_equal(ra["stats"], rb["stats"])
    finally:
        a.close()
        b.close()
