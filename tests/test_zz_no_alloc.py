"""dade_search_noalloc: the search entry point for callers that cannot
allocate device memory at search time (an application whose allocator holds
all of the GPU's memory, or a path that cannot afford cudaMalloc's implicit
synchronisation).  Its scratch is a fixed 64 MiB device array inside the
library.  It must return what dade_search returns, bit for bit, call after
call, allocate nothing, refuse work that does not fit its scratch, and fail
with the same status as dade_search on invalid arguments.

This file is collected last (its name), so a run that stops at the first
failure has run every other test before it; it also passes alone."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch

    from paper_2404_16322_gb300 import build
    build.build()
    import paper_2404_16322_gb300 as G
    X, Q, T, cfg = synth.workload("tiny", n_train=500)
    mean, R, _ = G.dade_train_rotation(X)
    idx = G.ivf_build(X, mean, R, cfg["nlist"], kmeans_iters=5, seed=2)
    G.dade_fit_correction(idx, T, 10, 8, 16)
    yield G, idx, Q, torch
    idx.close()


def _buffers(torch, Q, K=10, P=8):
    dev = torch.device("cuda")
    B = len(Q)
    return dict(q=torch.from_numpy(np.ascontiguousarray(Q)).to(dev),
                k=torch.full((B,), K, dtype=torch.int32, device=dev),
                n=torch.full((B,), P, dtype=torch.int32, device=dev),
                ids=torch.full((B * K,), -7, dtype=torch.int64, device=dev),
                d=torch.full((B * K,), -7.0, dtype=torch.float32, device=dev),
                st=torch.zeros(1, dtype=torch.int32, device=dev))


def _run(torch, fn, idx, b, B, K=10, P=8, delta_d=16):
    fn(idx, b["q"], b["k"], b["n"], delta_d, b["ids"], b["d"], max_K=K, max_nprobe=P, status=b["st"])
    torch.cuda.synchronize()
    assert int(b["st"].item()) == 0
    return b["ids"].view(B, K).cpu().numpy().copy(), b["d"].view(B, K).cpu().numpy().copy()


def test_noalloc_matches_dade_search_on_two_calls_in_a_row(setup):
    G, idx, Q, torch = setup
    # two different batches back to back: the second call must not see the
    # first call's leftovers in the shared scratch
    for part in (Q[:60], Q[40:]):
        b = _buffers(torch, part)
        got_i, got_d = _run(torch, G.dade_search_noalloc, idx, b, len(part))
        ref_i, ref_d = _run(torch, G.dade_search, idx, _buffers(torch, part), len(part))
        assert np.array_equal(got_i, ref_i)
        assert np.array_equal(got_d, ref_d)  # the same kernels on the same inputs: identical bits


def test_noalloc_allocates_nothing_on_a_fresh_index(setup):
    G, idx, Q, torch = setup
    X, _, T, cfg = synth.workload("tiny", n_train=300)
    mean, R, _ = G.dade_train_rotation(X)
    fresh = G.ivf_build(X, mean, R, cfg["nlist"], kmeans_iters=3, seed=4)
    try:
        G.dade_fit_correction(fresh, T, 10, 8, 16)
        b = _buffers(torch, Q)
        # one call loads the library's module (and with it the static array)
        _run(torch, G.dade_search_noalloc, idx, _buffers(torch, Q), len(Q))
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        # the fresh index has never been searched: a fallback to its own
        # per-stream scratch would allocate now and keep the memory
        first = _run(torch, G.dade_search_noalloc, fresh, b, len(Q))
        second = _run(torch, G.dade_search_noalloc, fresh, b, len(Q))
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        assert np.array_equal(first[0], second[0]) and np.array_equal(first[1], second[1])
        ref = _run(torch, G.dade_search, fresh, _buffers(torch, Q), len(Q))
        assert np.array_equal(first[0], ref[0]) and np.array_equal(first[1], ref[1])
    finally:
        fresh.close()


def test_noalloc_rejects_searches_larger_than_its_scratch(setup):
    from paper_2404_16322_gb300 import _lib
    G, idx, Q, torch = setup
    B = 50_000
    need = G.dade_search_workspace_size(idx, B, 16, 10, 8)
    assert need > 64 << 20
    dev = torch.device("cuda")
    q = torch.zeros((B, Q.shape[1]), dtype=torch.float32, device=dev)
    k = torch.full((B,), 10, dtype=torch.int32, device=dev)
    n = torch.full((B,), 8, dtype=torch.int32, device=dev)
    ids = torch.empty(B * 10, dtype=torch.int64, device=dev)
    d = torch.empty(B * 10, dtype=torch.float32, device=dev)
    with pytest.raises(_lib.DadeError) as e:
        G.dade_search_noalloc(idx, q, k, n, 16, ids, d, max_K=10, max_nprobe=8)
    assert e.value.status == 1 and "scratch" in str(e.value)


def test_noalloc_reports_the_same_status_as_dade_search(setup):
    from paper_2404_16322_gb300 import _lib
    G, idx, Q, torch = setup
    b = _buffers(torch, Q[:8])
    for kw in (dict(delta_d=32), dict(delta_d=12)):  # no table for 32 (ESTATE); 12 is not a step width
        errs = []
        for fn in (G.dade_search, G.dade_search_noalloc):
            with pytest.raises(_lib.DadeError) as e:
                fn(idx, b["q"], b["k"], b["n"], kw["delta_d"], b["ids"], b["d"], max_K=10, max_nprobe=8)
            errs.append((e.value.status, str(e.value)))
        assert errs[0] == errs[1]
    assert errs[0][0] == 1
