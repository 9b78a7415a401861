"""Serving: continuous batching of uneven requests over the C ABI.  Each
request's result must be the same when it is served alone as when it is
served in a mix of other requests (the wave schedule makes a query's result
independent of its batch), and batches must respect the memory budget."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served():
    from paper_2404_16322_gb300 import build
    build.build()
    import paper_2404_16322_gb300 as G
    X, Q, T, cfg = synth.workload("tiny", n_train=500, n_queries=300)
    mean, R, _ = G.dade_train_rotation(X)
    idx = G.ivf_build(X, mean, R, cfg["nlist"], kmeans_iters=5, seed=4)
    G.dade_fit_correction(idx, T, 10, 8, 16)
    yield G, idx, Q
    idx.close()


def _alone(G, idx, q, K, nprobe, max_K, max_nprobe):
    import torch
    dev = torch.device("cuda")
    ids = torch.empty(max_K, dtype=torch.int64, device=dev)
    d = torch.empty(max_K, dtype=torch.float32, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    G.dade_search(idx, torch.from_numpy(q[None, :]).to(dev), torch.tensor([K], dtype=torch.int32, device=dev),
                  torch.tensor([nprobe], dtype=torch.int32, device=dev), 16, ids, d, max_K=max_K,
                  max_nprobe=max_nprobe, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return ids.cpu().numpy()[:K], d.cpu().numpy()[:K]


@pytest.mark.parametrize("use_graphs", [True, False])
def test_results_same_alone_and_in_the_mix(served, use_graphs):
    from paper_2404_16322_gb300 import serving
    G, idx, Q = served
    rng = np.random.default_rng(11)
    n = len(Q)
    Ks = rng.choice([1, 10, 20], n)
    nps = rng.integers(1, 17, n)
    arr = serving.poisson_arrivals(n, rate=20_000, seed=3)
    reqs = [serving.Request(Q[i], int(Ks[i]), int(nps[i]), float(arr[i])) for i in range(n)]
    srv = serving.Server(G, idx, 16, max_K=20, max_nprobe=16, buckets=(8, 32, 128), slots=3,
                         use_graphs=use_graphs)
    out = srv.serve(reqs, max_batch=128)
    assert out["status"] == 0 and out["requests"] == n
    assert out["p99_ms"] >= out["p50_ms"] > 0
    for i in range(0, n, 7):
        ids, d = _alone(G, idx, Q[i], int(Ks[i]), int(nps[i]), 20, 16)
        assert np.array_equal(reqs[i].ids, ids)
        assert np.array_equal(reqs[i].dists, d)


def test_memory_budget_limits_batch_size(served):
    from paper_2404_16322_gb300 import serving
    G, idx, Q = served
    buckets = (8, 32, 128)
    ws = {b: G.dade_search_workspace_size(idx, b, 16, 10, 8) for b in buckets}
    budget = ws[32] + ws[8]  # room for one 32-query batch plus one 8-query batch
    srv = serving.Server(G, idx, 16, max_K=10, max_nprobe=8, buckets=buckets, slots=2, mem_budget=budget,
                         use_graphs=False)
    reqs = [serving.Request(Q[i], 10, 8, 0.0) for i in range(200)]
    out = srv.serve(reqs, max_batch=128)
    assert out["status"] == 0 and out["requests"] == 200
    assert out["mean_batch"] <= 32
    assert all(r.ids is not None and len(r.ids) == 10 for r in reqs)


def test_two_indices_share_the_arena(served):
    """Two resident indices of different dimension behind one server: each
    request's result equals its search alone on its own index, and the
    arena is empty again afterwards."""
    import torch
    from paper_2404_16322_gb300 import serving
    G, idx, Q = served
    X2, Q2, T2, cfg2 = synth.workload("tiny", n_train=400, n_queries=200)
    X2, Q2, T2 = X2[:, :64].copy(), Q2[:, :64].copy(), T2[:, :64].copy()
    mean, R, _ = G.dade_train_rotation(X2)
    idx2 = G.ivf_build(X2, mean, R, 32, kmeans_iters=4, seed=5, dtype="bf16")
    try:
        G.dade_fit_correction(idx2, T2, 10, 8, 16)
        tenants = [serving.Tenant(idx, 16, 20, 16, first_wave=2, wave_growth_log2=30),
                   serving.Tenant(idx2, 16, 20, 16, first_wave=2, wave_growth_log2=30)]
        srv = serving.Server(G, tenants, buckets=(8, 32, 128), slots=3, use_graphs=False)
        rng = np.random.default_rng(2)
        n = 400
        ten = rng.integers(0, 2, n)
        qi = rng.integers(0, 200, n)
        ks = rng.choice([1, 10, 20], n)
        nps = rng.integers(1, 17, n)
        arr = serving.poisson_arrivals(n, rate=30_000, seed=9)
        ids, d, done, out = srv.serve_pool([Q[:200], Q2], ten, qi, ks, nps, arr, max_batch=128)
        assert out["status"] == 0 and out["requests"] == n and set(out["tenants"]) == {0, 1}
        assert srv.arena.used == 0
        dev = torch.device("cuda")
        for i in range(0, n, 9):
            t = tenants[ten[i]]
            q = (Q if ten[i] == 0 else Q2)[qi[i]]
            oi = torch.empty(20, dtype=torch.int64, device=dev)
            od = torch.empty(20, dtype=torch.float32, device=dev)
            G.dade_search(t.idx, torch.from_numpy(q[None, :]).to(dev),
                          torch.tensor([ks[i]], dtype=torch.int32, device=dev),
                          torch.tensor([nps[i]], dtype=torch.int32, device=dev), 16, oi, od, max_K=20,
                          max_nprobe=16, first_wave=2, wave_growth_log2=30)
            torch.cuda.synchronize()
            k = int(ks[i])
            assert np.array_equal(ids[i, :k], oi.cpu().numpy()[:k])
            assert np.array_equal(d[i, :k], od.cpu().numpy()[:k])
    finally:
        idx2.close()
