"""Bucket-sharded search, host side: the library's bucket partition (through
the C ABI, no device needed) and the one exchange step (all_gather of the
ranks' top-K lists) over gloo with two ranks on CPU, checked against the
oracle: the merged per-shard exact results equal the unsharded result."""
import os

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import paper_2404_16322_gb300 as G
from oracle import ivf, search


@pytest.mark.parametrize("n_shards", [1, 2, 3, 7])
def test_partition_covers_and_balances(n_shards):
    rng = np.random.default_rng(n_shards)
    sizes = rng.integers(0, 500, 64)
    own = G.dade_shard_owners(sizes, n_shards)
    assert own.shape == (64,) and own.min() >= 0 and own.max() < n_shards
    loads = np.bincount(own, weights=sizes, minlength=n_shards)
    # largest-first greedy: no shard exceeds another by more than one bucket
    assert loads.max() - loads.min() <= sizes.max()
    assert np.array_equal(own, G.dade_shard_owners(sizes, n_shards))  # deterministic


def test_partition_edge_cases():
    sizes = np.array([4, 4, 4, 4])
    assert np.array_equal(G.dade_shard_owners(sizes, 1), np.zeros(4, np.int32))
    assert sorted(G.dade_shard_owners(sizes, 4).tolist()) == [0, 1, 2, 3]
    from paper_2404_16322_gb300 import _lib
    with pytest.raises(_lib.DadeError):
        G.dade_shard_owners(sizes, 5)
    with pytest.raises(_lib.DadeError):
        G.dade_shard_owners(np.array([3, -1]), 1)


def _small_index():
    rng = np.random.default_rng(31)
    D, N, nlist = 16, 1500, 12
    X = (rng.standard_normal((N, D)) * np.linspace(2, 0.3, D)).astype(np.float32)
    Q = (rng.standard_normal((20, D)) * np.linspace(2, 0.3, D)).astype(np.float32)
    C, _, _ = ivf.kmeans(X.astype(np.float64), np.arange(nlist), 3)
    a = ivf.assign(X.astype(np.float64), C)
    return X, Q, C, a, nlist


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from paper_2404_16322_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, Q, C, a, nlist = _small_index()
        own = shard.owners(np.bincount(a, minlength=nlist), world)
        rows = np.nonzero(own[a] == rank)[0]
        idx = search.OracleIndex(X[rows], np.zeros(X.shape[1]), np.eye(X.shape[1]), C, a[rows], dtype="f64",
                                 ids=rows)
        full = search.OracleIndex(X, np.zeros(X.shape[1]), np.eye(X.shape[1]), C, a, dtype="f64")
        probes = full.probe(full.rotate_queries(Q), 5)
        tabs = search.disabled_tables(search.n_steps(X.shape[1], 8))
        ids, d, _ = search.search(idx, Q, probes, 5, 10, 8, *tabs)
        ids_all, d_all = shard.gather_parts(torch.from_numpy(ids), torch.from_numpy(d.astype(np.float32)))
        if rank == 0:
            ref_i, ref_d, _ = search.search(full, Q, probes, 5, 10, 8, *tabs)
            out.put((ids_all.numpy(), d_all.numpy(), ref_i, ref_d.astype(np.float32)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gather_and_merge_equal_unsharded():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    ids_all, d_all, ref_i, ref_d = q.get(timeout=120)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert ids_all.shape == (2,) + ref_i.shape
    # merge the two ranks' lists by (distance, id): the unsharded result
    for b in range(ref_i.shape[0]):
        i = ids_all[:, b].ravel()
        d = d_all[:, b].ravel()
        ok = i >= 0
        o = np.lexsort((i[ok], d[ok]))[:10]
        assert np.array_equal(i[ok][o], ref_i[b]) and np.array_equal(d[ok][o], ref_d[b])
    # the two shards found disjoint candidates
    s0, s1 = set(ids_all[0][ids_all[0] >= 0].tolist()), set(ids_all[1][ids_all[1] >= 0].tolist())
    assert not (s0 & s1)


def _failing_rank(rank, world, port, out):
    # rank 1 fails before the exchange (a shard that cannot search); rank 0
    # must see an error from the gather within the group's timeout, not hang
    import datetime
    import time
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from paper_2404_16322_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(3)
    t0 = time.time()
    try:
        shard.gather_parts(torch.zeros((4, 10), dtype=torch.int64), torch.zeros((4, 10)))
        out.put(("no error", time.time() - t0))
    except Exception as e:  # the backend's error type differs across versions
        out.put((type(e).__name__, time.time() - t0))


def test_a_failed_rank_surfaces_as_an_error_on_the_others():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29700 + os.getpid() % 1000
    ps = [ctx.Process(target=_failing_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    what, secs = q.get(timeout=120)
    for p in ps:
        p.join(timeout=60)
    assert what != "no error"
    assert secs < 60
    assert ps[1].exitcode == 3
