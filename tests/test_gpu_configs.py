"""GPU parity on the shapes of the other workloads, and the full-size SIFT
-shaped workload in the benchmark's launch configuration.

* GIST-shaped (D = 960, strong spectral decay, BF16 slabs, Delta_d = 32) and
  vMF-shaped (D = 96, L2-normalised, FP8 slabs, uneven K and nprobe) at
  sizes the oracle finishes in seconds, with the oracle's rotation, buckets
  and tables on both sides (pre-rotated: strict id parity).
* SIFT-shaped 1M x 128, 10k queries, nprobe 64, K 100, Delta_d 16, first
  wave 8 and one later wave -- the configuration bench.py selects and times
  -- against the oracle on 1,000 queries (the oracle given the library's
  rotation, centroids, assignment and tables), and on sampled queries
  through properties that hold at any size:
  returned distances are the exact distances of the returned ids (integer
  data: bit-exact in FP32), results are sorted and unique, every result of
  the pruned search that beats the full scan's K-th is in the full scan's
  result, and recall@10 against brute force on the sample.
* GIST-shaped 1M x 960 with BF16 slabs, 1,000 queries, nprobe 128, first
  wave 16 (the GIST-shaped bench configuration) against the oracle in the
  same way, and the 10M x 96 vMF-like
  set with BF16 and FP8 slabs and all 20,000 requests (K in [1, 100],
  nprobe in [8, 256]) in one call, also replayed from a CUDA graph, checked
  the same way (distances within 1e-5 of FP64)."""
import numpy as np
import pytest

import synth
from oracle import search

from . import gpu_helpers as H
from . import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2404_16322_gb300 import build
    build.build()
    import paper_2404_16322_gb300 as G
    return G


def _oracle_search(inp, Q, K, nprobe, delta_d, amb="exact", final_rel=np.inf):
    oidx = inp["oidx"]
    P = int(np.max(nprobe))
    pr = oidx.probe(oidx.rotate_queries(Q), P)
    ids, d, st, ad = search.search(oidx, Q, pr, nprobe, K, delta_d, inp["m1"].astype(np.float64),
                                   inp["beta"].astype(np.float64), amb=H.AMB[amb], final_rel=final_rel, with_amb=True, norm_eps=H.NORM_EPS)
    return ids, d, st, pr, ad


def test_gist_shaped_bf16_slabs(G):
    spec = synth.MixtureSpec(D=960, n_comp=32, alpha=1.3)
    X, Q, T = spec.sample(20_000, 1), spec.sample(60, 2), spec.sample(300, 3)
    inp = H.oracle_inputs(X, T, 64, iters=4, K=100, nprobe=8, delta_d=32, dtype="bf16", n_train=300,
                          prerotate=True)
    idx = H.build_gpu(G, None, inp, 64, dtype="bf16", delta_d=32)
    Qr = inp["rot"](Q)
    for final in (False, True):
        ids, d, st, pr, ad = _oracle_search(inp, Qr, 100, 8, 32, final_rel=search.FINAL_REL if final else np.inf)
        out = H.gpu_search(G, idx, Qr, 100, 8, 32, probe_in=pr, final_test=final, want=("stats",))
        parity.check(out["ids"], out["dists"], ids, d, inp["X"], Qr, 100, amb_d=ad)
        un = st[:, 4] == 0
        assert np.array_equal(out["stats"][un], st[un, :4])
        assert st[:, 1].sum() > 0
    idx.close()


def test_vmf_shaped_fp8_slabs_uneven_requests(G):
    spec = synth.VmfSpec(D=96, n_comp=64)
    X, Q, T = spec.sample(20_000, 1), spec.sample(120, 2), spec.sample(400, 3)
    inp = H.oracle_inputs(X, T, 64, iters=4, K=50, nprobe=12, delta_d=16, dtype="fp8", n_train=400,
                          prerotate=True)
    idx = H.build_gpu(G, None, inp, 64, dtype="fp8", delta_d=16)
    Qr = inp["rot"](Q)
    rng = np.random.default_rng(9)
    K = rng.integers(1, 101, len(Q)).astype(np.int32)
    npb = rng.integers(8, 17, len(Q)).astype(np.int32)
    for final in (False, True):
        ids, d, st, pr, ad = _oracle_search(inp, Qr, K, npb, 16, final_rel=search.FINAL_REL if final else np.inf)
        out = H.gpu_search(G, idx, Qr, K, npb, 16, probe_in=pr, max_K=100, max_nprobe=16, final_test=final,
                           want=("stats",))
        parity.check(out["ids"], out["dists"], ids, d, inp["X"], Qr, K, amb_d=ad)
        un = st[:, 4] == 0
        assert np.array_equal(out["stats"][un], st[un, :4])
    idx.close()


@pytest.fixture(scope="module")
def sift_full(G):
    X, Q, T, cfg = synth.workload("sift1m")
    mean, R, _ = G.dade_train_rotation(X, sample_n=1_000_000, seed=1)
    idx = G.ivf_build(X, mean, R, cfg["nlist"], kmeans_iters=10, seed=1, dtype="f32")
    G.dade_fit_correction(idx, T, 100, 64, 16, target_recall=0.995, seed=1)
    yield dict(X=X, Q=Q, idx=idx, mean=mean, R=R)
    idx.close()


def _library_oracle(G, idx, X, mean, R, dtype):
    """An oracle index on the library's instance: its rotation (mean, R),
    centroids and bucket assignment.  The oracle rotates, stores, estimates,
    tests and merges on its own in FP64; its rounding model allows the
    device's rotation to stray by H.FLIP_EPS * ||x'|| per coordinate."""
    C = G.dade_index_centroids(idx).astype(np.float64)
    a = G.dade_index_assignment(idx)
    return search.OracleIndex(X, mean, R, C, a, dtype=dtype, flip_eps=H.FLIP_EPS)


def _rotation_within_model(G, idx, oidx, qrot, Q, rows):
    """The device's rotated queries and (FP32 slabs) stored vectors stray
    from the FP64 rotation by less than the oracle's model assumes."""
    qr = oidx.rotate_queries(Q)
    q_err = np.abs(qrot - qr).max(axis=1) / np.linalg.norm(qr, axis=1)
    assert q_err.max() < H.FLIP_EPS, q_err.max()
    if oidx.dtype == "f32":
        xs = G.dade_index_stored(idx, rows.start, len(rows)).astype(np.float64)
        xr = oidx.Xs[rows]
        dev = np.abs(xs - xr)
        assert np.all(dev <= oidx.Xdev[rows]), (dev / oidx.Xdev[rows]).max()
    return float(q_err.max())


def _probes_within_near_ties(oidx, Q, probes, P):
    """The device's probe lists equal the FP64 ones except where centroid
    distances tie within 1e-5; returns the fraction of identical lists."""
    Qr = oidx.rotate_queries(Q)
    own = oidx.probe(Qr, P)
    same = np.all(own == probes, axis=1)
    for b in np.flatnonzero(~same):
        d = ((oidx.C - Qr[b]) ** 2).sum(1)
        kth = d[own[b, P - 1]]
        for l in set(own[b].tolist()) ^ set(probes[b].tolist()):
            assert abs(d[l] - kth) <= 1e-5 * kth, (b, l)
    return float(same.mean())


def test_sift_full_size_matches_the_oracle(G, sift_full):
    """The benchmarked configuration (1M x 128 integer data, nlist 4096,
    nprobe 64, K 100, Delta_d 16, first wave 8 then one wave) against the
    oracle on 1,000 queries of the 10,000-query batch, given the library's
    rotation, centroids, assignment and fitted tables.  Exact distances are
    integers (exact in FP32), so ids are compared at every rank below each
    query's first uncertain candidate, ties included, and distances bit for
    bit; work counters agree wherever no candidate is uncertain."""
    X, Q, idx = sift_full["X"], sift_full["Q"], sift_full["idx"]
    nq = 1000
    out = H.gpu_search(G, idx, Q, 100, 64, 16, first_wave=8, growth=30, want=("stats", "probes", "qrot"))
    assert out["status"] == 0
    oidx = _library_oracle(G, idx, X, sift_full["mean"], sift_full["R"], "f32")
    q_err = _rotation_within_model(G, idx, oidx, out["qrot"][:nq], Q[:nq], range(0, 20_000))
    same = _probes_within_near_ties(oidx, Q[:nq], out["probes"][:nq], 64)
    m1, beta = G.dade_get_correction(idx, 16)
    ids, d, st, ad = search.search(oidx, Q[:nq], out["probes"][:nq], 64, 100, 16, m1.astype(np.float64),
                                   beta.astype(np.float64), first_wave=8, growth=30, amb=H.AMB["f32"],
                                   with_amb=True, norm_eps=H.NORM_EPS, qdev_eps=H.FLIP_EPS)
    checked, total = parity.check(out["ids"][:nq], out["dists"][:nq], ids, d, X, Q[:nq], 100, amb_d=ad,
                                  exact_ties=True)
    un = st[:, 4] == 0
    assert np.array_equal(out["stats"][:nq, 0], st[:, 0])
    assert np.array_equal(out["stats"][:nq][un], st[un, :4])
    assert st[:, 1].sum() > 0.5 * st[:, 0].sum()
    print(f"SIFT_PARITY ranks_checked={checked}/{total} queries_certain={un.mean():.3f} "
          f"probe_lists_identical={same:.3f} rotation_err={q_err:.2e}")


def test_sift_full_size_in_the_benchmark_configuration(G, sift_full):
    X, Q, idx = sift_full["X"], sift_full["Q"], sift_full["idx"]
    pr = H.gpu_search(G, idx, Q, 100, 64, 16, first_wave=8, growth=30, want=("stats",))
    fu = H.gpu_search(G, idx, Q, 100, 64, 0, mode="full", first_wave=8, growth=30)
    assert pr["status"] == 0 and fu["status"] == 0
    sample = np.random.default_rng(5).choice(len(Q), 24, replace=False)
    Xd = X.astype(np.float64)
    hits = []
    for b in sample:
        q = Q[b].astype(np.float64)
        for out in (pr, fu):
            ids, dd = out["ids"][b], out["dists"][b]
            assert np.all(ids >= 0) and len(set(ids.tolist())) == 100
            ex = ((Xd[ids] - q) ** 2).sum(1)
            assert np.array_equal(dd.astype(np.float64), ex)  # integer data: exact
            assert np.all(np.diff(dd) >= 0)
        # pruning removes candidates only: whatever the full scan keeps below
        # its own K-th entry is found by the pruned search too, unless pruned
        kth = (fu["dists"][b][-1], fu["ids"][b][-1])
        better_p = {i for i, x in zip(pr["ids"][b], pr["dists"][b]) if (x, i) < kth}
        assert better_p <= set(fu["ids"][b].tolist())
        # brute-force recall@10 of the pruned search on the sample
        dall = ((Xd - q) ** 2).sum(1)
        gt = np.lexsort((np.arange(len(X)), dall))[:10]
        hits.append(len(set(gt.tolist()) & set(pr["ids"][b][:10].tolist())) / 10)
    assert np.mean(hits) >= 0.9
    st = pr["stats"]
    assert st[:, 1].sum() > 0.5 * st[:, 0].sum()  # most candidates are pruned



def _check_sampled(X, Q, pr, fu, K, sample, exact_bits=False):
    """Properties of the pruned (pr) and full-scan (fu) results on sampled
    queries; returns the brute-force recall@10 of the pruned search."""
    hits = []
    for b in sample:
        k = int(K[b])
        q = Q[b].astype(np.float64)
        for out in (pr, fu):
            ids, dd = out["ids"][b][:k], out["dists"][b][:k]
            v = ids >= 0
            assert len(set(ids[v].tolist())) == v.sum() and np.all(np.diff(dd[v]) >= 0)
            assert np.all(out["ids"][b][k:] == -1)
            ex = ((X[ids[v]].astype(np.float64) - q) ** 2).sum(1)
            if exact_bits:
                assert np.array_equal(dd[v].astype(np.float64), ex)
            else:
                assert np.all(np.abs(dd[v] - ex) <= 1e-5 * np.maximum(ex, 1e-3 * np.median(ex)))
        kth = (fu["dists"][b][k - 1], fu["ids"][b][k - 1])
        better_p = {i for i, x in zip(pr["ids"][b][:k], pr["dists"][b][:k]) if i >= 0 and (x, i) < kth}
        assert better_p <= set(fu["ids"][b][:k].tolist())
        if k >= 10:
            dall = np.empty(len(X))
            for c0 in range(0, len(X), 1 << 20):
                xc = X[c0:c0 + (1 << 20)].astype(np.float64)
                dall[c0:c0 + len(xc)] = ((xc - q) ** 2).sum(1)
            gt = np.lexsort((np.arange(len(X)), dall))[:10]
            hits.append(len(set(gt.tolist()) & set(pr["ids"][b][:10].tolist())) / 10)
    return float(np.mean(hits)) if hits else 1.0


def test_gist_full_size_in_the_benchmark_configuration(G):
    """GIST-shaped 1M x 960 with BF16 slabs, the benchmarked configuration
    (nprobe 128, K 100, Delta_d 16, first wave 16 then one wave), all 1,000
    queries against the oracle given the library's rotation, centroids,
    assignment and tables (the oracle bounds where the device's BF16 values
    may round to the neighbouring value), plus the sampled properties."""
    X, Q, T, cfg = synth.workload("gist1m")
    mean, R, _ = G.dade_train_rotation(X, sample_n=200_000, seed=1)
    idx = G.ivf_build(X, mean, R, cfg["nlist"], kmeans_iters=10, seed=1, dtype="bf16")
    try:
        G.dade_fit_correction(idx, T, 100, 64, 16, target_recall=0.995, seed=1)
        pr = H.gpu_search(G, idx, Q, 100, 128, 16, first_wave=16, growth=30, want=("stats", "probes", "qrot"))
        fu = H.gpu_search(G, idx, Q, 100, 128, 0, mode="full", first_wave=16, growth=30)
        assert pr["status"] == 0 and fu["status"] == 0
        sample = np.random.default_rng(6).choice(len(Q), 12, replace=False)
        rec = _check_sampled(X, Q, pr, fu, np.full(len(Q), 100), sample)
        assert rec >= 0.9
        st = pr["stats"]
        assert st[:, 3].sum() < 0.3 * st[:, 0].sum() * X.shape[1]   # well under a full scan's dims
        oidx = _library_oracle(G, idx, X, mean, R, "bf16")
        q_err = _rotation_within_model(G, idx, oidx, pr["qrot"], Q, range(0))
        same = _probes_within_near_ties(oidx, Q, pr["probes"], 128)
        m1, beta = G.dade_get_correction(idx, 16)
        ids, d, ost, ad = search.search(oidx, Q, pr["probes"], 128, 100, 16, m1.astype(np.float64),
                                        beta.astype(np.float64), first_wave=16, growth=30, amb=H.AMB["f32"],
                                        with_amb=True, norm_eps=H.NORM_EPS, qdev_eps=H.FLIP_EPS)
        del oidx
        checked, total = parity.check(pr["ids"], pr["dists"], ids, d, X, Q, 100, amb_d=ad)
        un = ost[:, 4] == 0
        assert np.array_equal(st[:, 0], ost[:, 0])
        assert np.array_equal(st[un], ost[un, :4])
        print(f"GIST_PARITY ranks_checked={checked}/{total} queries_certain={un.mean():.3f} "
              f"probe_lists_identical={same:.3f} rotation_err={q_err:.2e}")
    finally:
        idx.close()


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_vmf_10m_full_size_uneven_requests(G, dtype):
    """Config 4 at its stated size: 10M x 96 L2-normalised vMF-like vectors,
    all 20,000 requests in one call with K uniform in [1, 100] and nprobe
    uniform in [8, 256], BF16 or FP8-E4M3 slabs.  The candidate buffer is
    bounded (the waves run in passes), and the search replays bit for bit
    from a CUDA graph.  Checked on sampled queries: exact distances of the
    returned ids, sorted unique results, containment in the full scan's
    result, brute-force recall@10."""
    import torch
    X, Q, T, cfg = synth.workload("vmf10m")
    mean, R, _ = G.dade_train_rotation(X, sample_n=1_000_000, seed=1)
    idx = G.ivf_build(X, mean, R, cfg["nlist"], kmeans_iters=10, seed=1, dtype=dtype)
    try:
        G.dade_fit_correction(idx, T, 100, 64, 16, target_recall=0.995, seed=1)
        B = len(Q)
        assert B == 20_000
        rng = np.random.default_rng(10)
        K = rng.integers(1, 101, B).astype(np.int32)
        npb = rng.integers(8, 257, B).astype(np.int32)
        kw = dict(max_K=100, max_nprobe=256, first_wave=8, growth=30)
        pr = H.gpu_search(G, idx, Q, K, npb, 16, want=("stats",), **kw)
        fu = H.gpu_search(G, idx, Q, K, npb, 0, mode="full", **kw)
        assert pr["status"] == 0 and fu["status"] == 0
        sample = np.random.default_rng(7).choice(B, 8, replace=False)
        rec = _check_sampled(X, Q, pr, fu, K, sample)
        assert rec >= 0.8
        st = pr["stats"]
        assert st[:, 1].sum() > 0.3 * st[:, 0].sum()
        # the same search captured in a CUDA graph and replayed
        dev = torch.device("cuda")
        q = torch.from_numpy(Q).to(dev)
        kt = torch.from_numpy(K).to(dev)
        nt = torch.from_numpy(npb).to(dev)
        ids = torch.full((B * 100,), -7, dtype=torch.int64, device=dev)
        d = torch.full((B * 100,), -7.0, dtype=torch.float32, device=dev)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        ws = torch.empty(G.dade_search_workspace_size(idx, B, 16, 100, 256, first_wave=8, wave_growth_log2=30),
                         dtype=torch.uint8, device=dev)
        assert ws.numel() < 12 << 30  # the candidate buffer is bounded, not B x the worst wave
        call = dict(max_K=100, max_nprobe=256, first_wave=8, wave_growth_log2=30, workspace=ws, status=status)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            G.dade_search(idx, q, kt, nt, 16, ids, d, **call)  # first call: kernel attributes set outside capture
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            G.dade_search(idx, q, kt, nt, 16, ids, d, **call)
        ids.fill_(-7)
        d.fill_(-7.0)
        graph.replay()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert np.array_equal(ids.view(B, 100).cpu().numpy(), pr["ids"])
        assert np.array_equal(d.view(B, 100).cpu().numpy(), pr["dists"])
    finally:
        idx.close()
