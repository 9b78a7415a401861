"""The top-nprobe bucket selection on the device, on 4096 centroids of
which every one has three exact duplicates, so that ties in distance are
exact and must be broken by the lower list id: the nprobe nearest are the
first nprobe of any larger selection (the order is a total order on
(distance, id)), and equal distances come out in increasing id order."""
import numpy as np
import pytest

from . import gpu_helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2404_16322_gb300 import build
    build.build()
    import paper_2404_16322_gb300 as G
    return G


@pytest.fixture(scope="module")
def dup_index(G):
    rng = np.random.default_rng(12)
    D, nlist = 16, 4096
    uniq = rng.standard_normal((nlist // 4, D)).astype(np.float32)
    C = np.repeat(uniq, 4, axis=0)                      # buckets 4u .. 4u + 3 share a centroid
    X = (C[rng.integers(0, nlist, 40000)] + 0.05 * rng.standard_normal((40000, D))).astype(np.float32)
    a = ((X[:, None, :].astype(np.float64) - C[None, :, :]) ** 2).sum(-1).argmin(1).astype(np.int32)
    idx = G.ivf_build(X, np.zeros(D), np.eye(D), nlist, centroids=C, assign=a)
    Q = rng.standard_normal((300, D)).astype(np.float32)
    yield dict(G=G, idx=idx, Q=Q, C=C, X=X)
    idx.close()


def _probes(G, s, nprobe):
    out = H.gpu_search(G, s["idx"], s["Q"], 1, nprobe, 0, mode="full", want=("probes",))
    assert out["status"] == 0
    return out["probes"]


def test_smaller_selections_are_prefixes_of_larger_ones(G, dup_index):
    ref = _probes(G, dup_index, 600)
    for np_ in (1, 7, 64, 200, 256):
        got = _probes(G, dup_index, np_)
        assert np.array_equal(got[:, :np_], ref[:, :np_]), np_


def test_ties_go_to_the_lower_list_id(G, dup_index):
    ref = _probes(G, dup_index, 600)
    C = dup_index["C"].astype(np.float64)
    for b in range(ref.shape[0]):
        p = ref[b]
        # the four copies of a centroid are adjacent, in increasing id order
        grp = p // 4
        for r in range(len(p) - 1):
            if grp[r] == grp[r + 1]:
                assert p[r] < p[r + 1]
        # the distances (FP64 recomputation) are non-decreasing up to FP32 rounding
        q = dup_index["Q"][b].astype(np.float64)
        d = ((C[p] - q) ** 2).sum(1)
        assert np.all(np.diff(d) >= -1e-4 * (1 + d[1:]))
