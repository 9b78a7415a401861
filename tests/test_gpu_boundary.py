"""The C-ABI boundary's conventions, on the GPU:

* one index searched concurrently on two streams (no caller workspace, so
  each stream uses the index's per-stream scratch) gives, on each stream,
  exactly the results of a serial search;
* the ragged output (out_offsets_dev: a prefix of per-query K, results
  packed back to back) holds, for every query, the oracle-checked result of
  the padded layout, and nothing is written outside the packed range;
* ivf_build from rows in device memory builds the same index as from host
  rows.
"""
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


@pytest.fixture(scope="module")
def pre(G):
    X, Q, T, cfg = synth.workload("tiny")
    inp = H.oracle_inputs(X, T, cfg["nlist"], K=10, nprobe=8, delta_d=16, prerotate=True)
    idx = H.build_gpu(G, None, inp, cfg["nlist"])
    yield dict(X=inp["X"], Q=inp["rot"](Q), inp=inp, idx=idx, cfg=cfg)
    idx.close()


def _dev(torch, a, dt):
    return torch.from_numpy(np.ascontiguousarray(a, dt)).cuda()


def test_two_streams_search_one_index_concurrently(G, pre):
    import torch
    idx, Q = pre["idx"], pre["Q"]
    rng = np.random.default_rng(3)
    # two different request mixes, searched many times over on two streams
    parts = []
    for s in range(2):
        B = 100
        q = Q[rng.integers(0, len(Q), B)] + rng.normal(scale=0.01, size=(B, Q.shape[1])).astype(np.float32)
        parts.append(dict(q=_dev(torch, q, np.float32), k=_dev(torch, rng.integers(1, 21, B), np.int32),
                          n=_dev(torch, rng.integers(1, 17, B), np.int32), B=B))
    ref = []
    for p in parts:  # serial reference on the default stream
        ids = torch.empty(p["B"] * 20, dtype=torch.int64, device="cuda")
        d = torch.empty(p["B"] * 20, dtype=torch.float32, device="cuda")
        G.dade_search(idx, p["q"], p["k"], p["n"], 16, ids, d, max_K=20, max_nprobe=16)
        torch.cuda.synchronize()
        ref.append((ids.cpu().numpy(), d.cpu().numpy()))
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [[(torch.empty(p["B"] * 20, dtype=torch.int64, device="cuda"),
              torch.empty(p["B"] * 20, dtype=torch.float32, device="cuda")) for _ in range(8)] for p in parts]
    status = [torch.zeros(1, dtype=torch.int32, device="cuda") for _ in parts]
    torch.cuda.synchronize()
    for r in range(8):  # interleaved enqueues: the streams' work overlaps on the device
        for s, p in enumerate(parts):
            with torch.cuda.stream(streams[s]):
                ids, d = outs[s][r]
                G.dade_search(idx, p["q"], p["k"], p["n"], 16, ids, d, max_K=20, max_nprobe=16,
                              status=status[s], stream=streams[s])
    torch.cuda.synchronize()
    for s in range(2):
        assert int(status[s].item()) == 0
        for r in range(8):
            assert np.array_equal(outs[s][r][0].cpu().numpy(), ref[s][0])
            assert np.array_equal(outs[s][r][1].cpu().numpy(), ref[s][1])


def test_ragged_packed_output_matches_the_oracle(G, pre):
    import torch
    idx, Q, X = pre["idx"], pre["Q"], pre["X"]
    B = len(Q)
    rng = np.random.default_rng(8)
    K = rng.integers(1, 31, B).astype(np.int32)
    K[::17] = 0  # inactive slots take no room
    npb = rng.integers(1, 17, B).astype(np.int32)
    oidx = pre["inp"]["oidx"]
    pr = oidx.probe(oidx.rotate_queries(Q), 16)
    off = np.zeros(B + 1, np.int64)
    np.cumsum(K, out=off[1:])
    total = int(off[-1])
    guard = 64
    ids = torch.full((total + guard,), -7, dtype=torch.int64, device="cuda")
    d = torch.full((total + guard,), -7.0, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    G.dade_search(idx, _dev(torch, Q, np.float32), _dev(torch, K, np.int32), _dev(torch, npb, np.int32), 16, ids, d,
                  max_K=30, max_nprobe=16, probe_in=_dev(torch, pr, np.int32), status=st,
                  offsets=_dev(torch, off, np.int64))
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ids, d = ids.cpu().numpy(), d.cpu().numpy()
    assert np.all(ids[total:] == -7) and np.all(d[total:] == -7.0)  # nothing past the packed range
    # unpack to the padded layout and compare with the oracle, rank by rank
    gi = np.full((B, 30), -1, np.int64)
    gd = np.full((B, 30), np.inf, np.float32)
    for b in range(B):
        gi[b, :K[b]] = ids[off[b]:off[b + 1]]
        gd[b, :K[b]] = d[off[b]:off[b + 1]]
    live = K > 0
    Kq = np.maximum(K, 1)
    oi, od, ost, ad = search.search(oidx, Q[live], pr[live], npb[live], Kq[live], 16,
                                    pre["inp"]["m1"].astype(np.float64), pre["inp"]["beta"].astype(np.float64),
                                    amb=H.AMB["exact"], with_amb=True, norm_eps=H.NORM_EPS)
    parity.check(gi[live], gd[live], oi, od, X, Q[live], K[live], amb_d=ad)
    # the padded layout of the same search holds the same entries
    pad = H.gpu_search(G, idx, Q, K, npb, 16, probe_in=pr, max_K=30, max_nprobe=16)
    for b in range(B):
        assert np.array_equal(pad["ids"][b, :K[b]], gi[b, :K[b]])
        assert np.array_equal(pad["dists"][b, :K[b]], gd[b, :K[b]])


def test_ivf_build_from_device_rows(G):
    import torch
    X, Q, T, cfg = synth.workload("tiny", n_train=300)
    mean, R, _ = G.dade_train_rotation(X)
    a = G.ivf_build(X, mean, R, cfg["nlist"], kmeans_iters=4, seed=3, dtype="bf16")
    b = G.ivf_build(torch.from_numpy(X).cuda(), mean, R, cfg["nlist"], kmeans_iters=4, seed=3, dtype="bf16")
    try:
        assert np.array_equal(G.dade_index_assignment(a), G.dade_index_assignment(b))
        assert np.array_equal(G.dade_index_centroids(a), G.dade_index_centroids(b))
        assert np.array_equal(G.dade_index_stored(a), G.dade_index_stored(b))
        m1, beta = G.dade_fit_correction(a, T, 10, 8, 16, seed=1)
        G.dade_set_correction(b, 16, m1, beta)
        ra = H.gpu_search(G, a, Q, 10, 8, 16, want=("stats",))
        rb = H.gpu_search(G, b, Q, 10, 8, 16, want=("stats",))
        for k in ("ids", "dists", "stats"):
            assert np.array_equal(ra[k], rb[k]), k
        # the stored values are the slab precision's rounding of the rotated rows
        xs = G.dade_index_stored(a, 100, 50).astype(np.float64)
        xr = (X[100:150].astype(np.float64) - mean) @ R.T
        assert np.all(np.abs(xs - xr) <= 2.0 ** -8 * np.abs(xr) + 1e-5 * np.linalg.norm(xr, axis=1, keepdims=True))
    finally:
        a.close()
        b.close()


def test_kernel_count_of_a_search(G, pre):
    """dade_search_kernel_count captures the call without running it: the
    outputs stay untouched, and more passes mean more launches (one scan and
    one merge per pass)."""
    import torch
    idx, Q = pre["idx"], pre["Q"]
    B = len(Q)
    q = _dev(torch, Q, np.float32)
    k = torch.full((B,), 10, dtype=torch.int32, device="cuda")
    n = torch.full((B,), 8, dtype=torch.int32, device="cuda")
    ids = torch.full((B * 10,), -7, dtype=torch.int64, device="cuda")
    d = torch.full((B * 10,), -7.0, dtype=torch.float32, device="cuda")
    counts = {}
    for budget in (0, 1):
        kw = dict(max_K=10, max_nprobe=8, first_wave=1, wave_growth_log2=1, candidate_budget_bytes=budget)
        ws = torch.empty(G.dade_search_workspace_size(idx, B, 16, 10, 8, first_wave=1, wave_growth_log2=1,
                                                      candidate_budget_bytes=budget), dtype=torch.uint8,
                         device="cuda")
        counts[budget] = G.dade_search_kernel_count(idx, q, k, n, 16, ids, d, workspace=ws, **kw)
    torch.cuda.synchronize()
    assert np.all(ids.cpu().numpy() == -7)
    # waves of ranks [0,1) [1,2) [2,4) [4,8): 4 passes; one rank per pass: 8
    assert counts[1] - counts[0] == 2 * (8 - 4)
    assert counts[0] > 2 * 4
