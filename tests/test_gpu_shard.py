"""Bucket-sharded search on one GPU with virtual shards: shard indexes from
dade_index_shard hold exactly their buckets, and merging the shards' results
with dade_merge_topk gives the unsharded result when pruning is off (the
full-dimension scan); with pruning on every merged result is a valid top-K
of exact distances."""
import numpy as np
import pytest

import synth
from oracle import knn

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
def built(G):
    X, Q, T, cfg = synth.workload("tiny")
    mu, R, _ = G.dade_train_rotation(X)
    idx = G.ivf_build(X, mu, R, cfg["nlist"], kmeans_iters=4, seed=3)
    G.dade_fit_correction(idx, T[:500], 10, 8, 16)
    yield dict(X=X, Q=Q, idx=idx)
    idx.close()


def _merge(G, parts, K, max_K):
    import torch
    dev = torch.device("cuda")
    ids = torch.from_numpy(np.stack([p["ids"] for p in parts])).to(dev)
    d = torch.from_numpy(np.stack([p["dists"] for p in parts])).to(dev)
    k = torch.from_numpy(np.broadcast_to(np.asarray(K, np.int32), (ids.shape[1],)).copy()).to(dev)
    oi = torch.empty(ids.shape[1:], dtype=torch.int64, device=dev)
    od = torch.empty(ids.shape[1:], dtype=torch.float32, device=dev)
    G.dade_merge_topk(ids, d, k, oi, od, max_K=max_K)
    torch.cuda.synchronize()
    return oi.cpu().numpy(), od.cpu().numpy()


@pytest.mark.parametrize("n", [2, 3])
def test_shards_hold_their_buckets_and_merge_to_unsharded(G, built, n):
    idx, Q = built["idx"], built["Q"]
    sizes = G.dade_index_list_sizes(idx)
    own = G.dade_shard_owners(sizes, n)
    shards = [G.dade_index_shard(idx, n, s) for s in range(n)]
    for s, sh in enumerate(shards):
        assert np.array_equal(G.dade_index_list_sizes(sh), np.where(own == s, sizes, 0))
        assert G.dade_index_info_get(sh)["N"] == int(sizes[own == s].sum())
    ref = H.gpu_search(G, idx, Q, 10, 8, 0, mode="full")
    parts = [H.gpu_search(G, sh, Q, 10, 8, 0, mode="full") for sh in shards]
    mi, md = _merge(G, parts, 10, 10)
    assert np.array_equal(mi, ref["ids"]) and np.array_equal(md, ref["dists"])
    # pruned search per shard: valid merged top-K of exact distances, recall
    # against exact KNN close to the unsharded pruned search
    pp = [H.gpu_search(G, sh, Q, 10, 8, 16) for sh in shards]
    pi, pd = _merge(G, pp, 10, 10)
    X = built["X"]
    for b in range(len(Q)):
        assert len(set(pi[b].tolist())) == 10 and np.all(np.diff(pd[b]) >= 0)
        ex = ((X[pi[b]].astype(np.float64) - Q[b].astype(np.float64)) ** 2).sum(1)
        assert np.allclose(pd[b], ex, rtol=1e-5)
    gi, _ = knn.exact_knn(X, Q, 10)
    un = H.gpu_search(G, idx, Q, 10, 8, 16)
    assert parity.recall(pi, gi, 10) >= parity.recall(un["ids"], gi, 10) - 0.02
    for sh in shards:
        sh.close()


def test_merge_uneven_K_and_padding(G):
    import torch
    rng = np.random.default_rng(4)
    B, Km, P = 50, 16, 3
    K = rng.integers(0, Km + 1, B).astype(np.int32)
    parts = []
    for p in range(P):
        n = rng.integers(0, Km + 1, B)
        ids = np.full((B, Km), -1, np.int64)
        d = np.full((B, Km), np.inf, np.float32)
        for b in range(B):
            dd = np.sort(rng.integers(0, 40, n[b]).astype(np.float32))
            ids[b, :n[b]] = np.sort(rng.choice(1000, n[b], replace=False)) + 1000 * p
            o = np.lexsort((ids[b, :n[b]], dd))
            d[b, :n[b]] = dd[o]
            ids[b, :n[b]] = ids[b, :n[b]][o]
        parts.append(dict(ids=ids, dists=d))
    mi, md = _merge(G, parts, K, Km)
    for b in range(B):
        i = np.concatenate([p["ids"][b] for p in parts])
        d = np.concatenate([p["dists"][b] for p in parts])
        ok = i >= 0
        o = np.lexsort((i[ok], d[ok]))[:K[b]]
        want_i = np.full(Km, -1, np.int64)
        want_d = np.full(Km, np.inf, np.float32)
        want_i[:len(o)] = i[ok][o]
        want_d[:len(o)] = d[ok][o]
        assert np.array_equal(mi[b], want_i) and np.array_equal(md[b], want_d), b


def test_res_on_shards_with_a_frozen_tau_matches_unsharded(G, built):
    # the RES test of a (query, candidate) pair depends only on the pair,
    # the index-wide variances (shards keep their parent's) and tau: with one
    # frozen tau per query the shards' decisions are the unsharded ones
    idx, Q = built["idx"], built["Q"]
    ref = H.gpu_search(G, idx, Q, 10, 8, 0, mode="full", want=("probes",))
    tau = ref["dists"][:, 9].astype(np.float32)
    base = H.gpu_search(G, idx, Q, 10, 8, 16, probe_in=ref["probes"], tau=tau, estimator="res", res_m=1.0,
                        want=("stats",))
    shards = [G.dade_index_shard(idx, 2, s) for s in range(2)]
    parts = [H.gpu_search(G, sh, Q, 10, 8, 16, probe_in=ref["probes"], tau=tau, estimator="res", res_m=1.0,
                          want=("stats",)) for sh in shards]
    assert base["status"] == 0 and all(p["status"] == 0 for p in parts)
    assert np.array_equal(sum(p["stats"] for p in parts), base["stats"])
    assert base["stats"][:, 1].sum() > 0
    mi, md = _merge(G, parts, 10, 10)
    assert np.array_equal(mi, base["ids"]) and np.array_equal(md, base["dists"])
    for sh in shards:
        sh.close()
