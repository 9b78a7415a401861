"""dade_search_noalloc: the search entry point for callers that cannot
allocate device memory at search time (an application whose allocator holds
all of the GPU's memory, or a path that cannot afford cudaMalloc's implicit
synchronisation).  Its scratch is a fixed 64 MiB device array inside the
library.  It must return what dade_search returns, call after call, and
refuse work that does not fit its scratch."""
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


def _run(G, torch, idx, Q, fn):
    dev = torch.device("cuda")
    B, K, P = len(Q), 10, 8
    q = torch.from_numpy(np.ascontiguousarray(Q)).to(dev)
    k = torch.full((B,), K, dtype=torch.int32, device=dev)
    n = torch.full((B,), P, dtype=torch.int32, device=dev)
    ids = torch.full((B * K,), -7, dtype=torch.int64, device=dev)
    d = torch.full((B * K,), -7.0, dtype=torch.float32, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    fn(idx, q, k, n, 16, ids, d, max_K=K, max_nprobe=P, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return ids.view(B, K).cpu().numpy(), d.view(B, K).cpu().numpy()


def test_noalloc_matches_dade_search_on_two_calls_in_a_row(setup):
    G, idx, Q, torch = setup
    # two different batches back to back: the second call must not see the
    # first call's leftovers in the shared scratch
    for part in (Q[:60], Q[40:]):
        ref_i, ref_d = _run(G, torch, idx, part, G.dade_search)
        got_i, got_d = _run(G, torch, idx, part, G.dade_search_noalloc)
        assert np.array_equal(got_i, ref_i)
        assert np.allclose(got_d, ref_d, rtol=1e-5, atol=0)


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
