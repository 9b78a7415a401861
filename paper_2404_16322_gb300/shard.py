"""Bucket-sharded search across processes (one shard of the index per rank).

Every rank holds the index of its own buckets (``dade_index_shard``), runs
the whole search on its shard with the same queries, and the ranks' top-K
lists are gathered (``torch.distributed.all_gather``: the one exchange step
of the path, K x 12 bytes per query per rank) and merged by (distance, id)
with ``dade_merge_topk``.  A query probes the same buckets on every rank
because every shard keeps all centroids; waves and thresholds stay local to
a shard.  With pruning off the merged result equals the unsharded one.
"""
from __future__ import annotations

import numpy as np


def owners(list_sizes, n_shards: int) -> np.ndarray:
    """Owner shard of every bucket (the library's host partition)."""
    from . import dade_shard_owners
    return dade_shard_owners(list_sizes, n_shards)


def gather_parts(ids, dists, group=None):
    """All ranks' (B, K) results stacked as (world, B, K) tensors, in rank
    order (works with gloo on CPU tensors and NCCL on CUDA tensors)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    ids_all = [torch.empty_like(ids) for _ in range(world)]
    d_all = [torch.empty_like(dists) for _ in range(world)]
    dist.all_gather(ids_all, ids.contiguous(), group=group)
    dist.all_gather(d_all, dists.contiguous(), group=group)
    return torch.stack(ids_all), torch.stack(d_all)


def sharded_search(G, shard_index, Q, K, nprobe, delta_d: int, *, max_K: int, max_nprobe: int, group=None,
                   **search_kw):
    """This rank's search over its shard, then the gather and the merge; every
    rank returns the merged (ids, dists) as (B, max_K) CUDA tensors."""
    import torch
    B = Q.shape[0]
    ids = torch.empty(B * max_K, dtype=torch.int64, device=Q.device)
    dists = torch.empty(B * max_K, dtype=torch.float32, device=Q.device)
    G.dade_search(shard_index, Q, K, nprobe, delta_d, ids, dists, max_K=max_K, max_nprobe=max_nprobe,
                  **search_kw)
    ids_all, d_all = gather_parts(ids.view(B, max_K), dists.view(B, max_K), group)
    out_i = torch.empty((B, max_K), dtype=torch.int64, device=Q.device)
    out_d = torch.empty((B, max_K), dtype=torch.float32, device=Q.device)
    G.dade_merge_topk(ids_all, d_all, K, out_i, out_d, max_K=max_K)
    return out_i, out_d
