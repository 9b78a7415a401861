"""Continuous-batching search server over the C ABI, for one or several
resident indices (tenants).

Requests (one query vector, the index it targets, its K and nprobe) arrive
over time.  The server keeps the indices, the slots' I/O buffers and one
workspace arena resident on the device and runs a single scheduling loop:

* each tenant has a FIFO queue of arrived requests; a free *slot* serves the
  tenant whose oldest waiting request arrived first, taking up to
  ``max_batch`` of that tenant's waiting requests, padded to the smallest
  batch bucket that holds them with inactive queries (K = 0, nprobe = 0);
* admission by memory: the batch's dade_search workspace is a byte range of
  the arena (``dade_arena_*``: first fit, aligned, coalescing), allocated when
  the batch launches and released when it completes.  A batch whose
  workspace does not fit shrinks to a smaller bucket, or waits for a
  running batch to release its range;
* the slot copies its requests from pinned host memory, runs dade_search and
  copies the results back, all on its own stream, so batches of different
  slots overlap on the device.

With ``use_graphs`` each (slot, tenant, bucket, arena offset) is captured
once as a CUDA graph (copies, search, copies) the first time it is used and
replayed afterwards; captures are counted in the summary.

A query's result does not depend on the batch it travels in: the search's
wave schedule freezes each query's threshold per wave of its own probe
ranks, and every (query, candidate) distance is computed with the same
arithmetic whatever the batch.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np


@dataclasses.dataclass
class Request:
    query: np.ndarray        # (D,) float32
    K: int
    nprobe: int
    arrival: float = 0.0     # seconds from the start of serve()
    tenant: int = 0
    done: float = -1.0
    ids: np.ndarray | None = None
    dists: np.ndarray | None = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclasses.dataclass
class Tenant:
    """One resident index and the search configuration its requests use."""
    idx: object
    delta_d: int
    max_K: int
    max_nprobe: int
    mode: str = "prune"
    first_wave: int = 1
    wave_growth_log2: int = 0
    final_test: bool = False
    scan_kernel: str = "auto"
    queries_per_unit: int = 0


class _Slot:
    def __init__(self, torch, B, D, K):
        dev = torch.device("cuda")
        self.stream = torch.cuda.Stream()
        self.q_h = torch.zeros(B * D, dtype=torch.float32).pin_memory()
        self.k_h = torch.zeros(B, dtype=torch.int32).pin_memory()
        self.n_h = torch.zeros(B, dtype=torch.int32).pin_memory()
        self.ids_h = torch.empty(B * K, dtype=torch.int64).pin_memory()
        self.d_h = torch.empty(B * K, dtype=torch.float32).pin_memory()
        self.q = torch.zeros(B * D, dtype=torch.float32, device=dev)
        self.k = torch.zeros(B, dtype=torch.int32, device=dev)
        self.n = torch.zeros(B, dtype=torch.int32, device=dev)
        self.ids = torch.empty(B * K, dtype=torch.int64, device=dev)
        self.d = torch.empty(B * K, dtype=torch.float32, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.event = torch.cuda.Event()
        self.graphs = {}
        self.batch = None  # (tenant, request positions, bucket, arena offset)


class Server:
    """Server(G, tenants, ...) with a list of Tenant; or, for one index,
    Server(G, idx, delta_d, max_K=..., max_nprobe=..., mode=..., first_wave=...,
    wave_growth_log2=..., final_test=...)."""

    def __init__(self, G, tenants, delta_d: int | None = None, max_K: int = 0, max_nprobe: int = 0,
                 buckets=(16, 64, 256, 1024), slots: int = 2, mem_budget: int | None = None,
                 use_graphs: bool = True, mode: str = "prune", first_wave: int = 1, wave_growth_log2: int = 0,
                 final_test: bool = False, align: int = 4096):
        import torch
        if not isinstance(tenants, (list, tuple)):
            tenants = [Tenant(tenants, delta_d, max_K, max_nprobe, mode, first_wave, wave_growth_log2, final_test)]
        self.torch, self.G, self.tenants = torch, G, list(tenants)
        self.D = [G.dade_index_info_get(t.idx)["D"] for t in self.tenants]
        self.max_K = max(t.max_K for t in self.tenants)
        self.buckets = sorted(buckets)
        self.ws_of = {}
        for ti, t in enumerate(self.tenants):
            for b in self.buckets:
                self.ws_of[ti, b] = G.dade_search_workspace_size(
                    t.idx, b, t.delta_d, t.max_K, t.max_nprobe, mode=t.mode, first_wave=t.first_wave,
                    wave_growth_log2=t.wave_growth_log2, final_test=t.final_test, scan_kernel=t.scan_kernel,
                    queries_per_unit=t.queries_per_unit) + 256
        ws_max = max(self.ws_of.values())
        self.mem_budget = mem_budget if mem_budget is not None else slots * (ws_max + align)
        self.arena = G.Arena(self.mem_budget, align)
        for ti in range(len(self.tenants)):  # every tenant's smallest batch must fit the empty arena
            need = -(-self.ws_of[ti, self.buckets[0]] // align) * align
            if need > self.arena.size:
                raise ValueError(f"memory budget {self.mem_budget} below tenant {ti}'s smallest batch workspace "
                                 f"({need} bytes)")
        self.arena_dev = torch.empty(self.arena.size + 256, dtype=torch.uint8, device="cuda")
        Bmax = self.buckets[-1]
        self.slots = [_Slot(torch, Bmax, max(self.D), self.max_K) for _ in range(slots)]
        self.use_graphs = use_graphs
        self.captures = 0
        # first launch of every kernel configuration outside any timing or capture
        for ti in range(len(self.tenants)):
            for b in self.buckets:
                s = self.slots[0]
                off = self.arena.alloc(self.ws_of[ti, b])
                if off < 0:
                    continue
                s.k_h[:b] = 0
                s.n_h[:b] = 0
                with torch.cuda.stream(s.stream):
                    self._enqueue(s, ti, b, off)
                s.stream.synchronize()
                self.arena.free(off)
        torch.cuda.synchronize()

    # ------------------------------------------------------------ device work
    def _workspace(self, off, nbytes):
        base = self.arena_dev.data_ptr() + off
        pad = (-base) % 256
        return self.arena_dev[off + pad: off + nbytes]

    def _enqueue(self, s: _Slot, ti: int, b: int, off: int):
        """H2D copies, the search over the first b rows, D2H copies."""
        t, D, K = self.tenants[ti], self.D[ti], self.tenants[ti].max_K
        s.q[: b * D].copy_(s.q_h[: b * D], non_blocking=True)
        s.k[:b].copy_(s.k_h[:b], non_blocking=True)
        s.n[:b].copy_(s.n_h[:b], non_blocking=True)
        self.G.dade_search(t.idx, s.q[: b * D].view(b, D), s.k[:b], s.n[:b], t.delta_d, s.ids, s.d, max_K=K,
                           max_nprobe=t.max_nprobe, mode=t.mode, first_wave=t.first_wave, status=s.status,
                           workspace=self._workspace(off, self.ws_of[ti, b]),
                           stream=self.torch.cuda.current_stream(), wave_growth_log2=t.wave_growth_log2,
                           final_test=t.final_test, scan_kernel=t.scan_kernel, queries_per_unit=t.queries_per_unit)
        s.ids_h[: b * K].copy_(s.ids[: b * K], non_blocking=True)
        s.d_h[: b * K].copy_(s.d[: b * K], non_blocking=True)

    def _launch(self, s: _Slot, ti: int, pos: np.ndarray, bucket: int, off: int):
        n, D = len(pos), self.D[ti]
        s.q_h.numpy()[: n * D] = self._pool[ti][self._qi[pos]].reshape(-1)
        s.k_h.numpy()[:n] = self._K[pos]
        s.n_h.numpy()[:n] = self._NP[pos]
        if bucket > n:
            s.k_h.numpy()[n:bucket] = 0
            s.n_h.numpy()[n:bucket] = 0
        torch = self.torch
        with torch.cuda.stream(s.stream):
            if self.use_graphs:
                key = (ti, bucket, off)
                g = s.graphs.get(key)
                if g is None:
                    g = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(g, stream=s.stream):
                        self._enqueue(s, ti, bucket, off)
                    s.graphs[key] = g
                    self.captures += 1
                g.replay()
            else:
                self._enqueue(s, ti, bucket, off)
            s.event.record(s.stream)
        s.batch = (ti, pos, bucket, off)

    def _finish(self, s: _Slot, now: float):
        ti, pos, bucket, off = s.batch
        n, K = len(pos), self.tenants[ti].max_K
        self._ids[pos, :K] = s.ids_h.numpy()[: n * K].reshape(n, K)
        self._dists[pos, :K] = s.d_h.numpy()[: n * K].reshape(n, K)
        self._done[pos] = now
        self.arena.free(off)
        s.batch = None

    def _admit(self, ti: int, n: int):
        """(bucket, arena offset) for up to n requests of tenant ti, or None."""
        bucket = next((b for b in self.buckets if b >= n), self.buckets[-1])
        while True:
            off = self.arena.alloc(self.ws_of[ti, bucket])
            if off >= 0:
                return bucket, off
            i = self.buckets.index(bucket)
            if i == 0:
                return None
            bucket = self.buckets[i - 1]

    # ------------------------------------------------------------ loop
    def serve_pool(self, pools, tenant, qidx, K, nprobe, arrival, max_batch: int = 1024):
        """Serve requests given as arrays: request i asks tenant[i] for
        pools[tenant[i]][qidx[i]] with K[i] and nprobe[i], arriving at
        arrival[i] seconds.  Returns (ids [n, max K], dists, done times [n],
        summary)."""
        self._pool = [np.ascontiguousarray(p, np.float32) for p in pools]
        self._qi = np.asarray(qidx, np.int64)
        self._K = np.asarray(K, np.int32)
        self._NP = np.asarray(nprobe, np.int32)
        ten = np.asarray(tenant, np.int64)
        arr = np.asarray(arrival, np.float64)
        n_all = len(arr)
        self._ids = np.full((n_all, self.max_K), -1, np.int64)
        self._dists = np.full((n_all, self.max_K), np.inf, np.float32)
        self._done = np.full(n_all, -1.0)
        # per tenant: its requests in arrival order
        order = [np.flatnonzero(ten == ti)[np.argsort(arr[ten == ti], kind="stable")]
                 for ti in range(len(self.tenants))]
        t_arr = [arr[o] for o in order]
        head = [0] * len(self.tenants)
        done = 0
        sizes, waits_mem = [], 0
        t0 = time.perf_counter()
        while done < n_all:
            now = time.perf_counter() - t0
            for s in self.slots:
                if s.batch is not None and s.event.query():
                    done += len(s.batch[1])
                    self._finish(s, time.perf_counter() - t0)
            arrived = [int(np.searchsorted(t_arr[ti], now, side="right")) for ti in range(len(self.tenants))]
            blocked = set()
            for s in self.slots:
                if s.batch is not None:
                    continue
                ready = [ti for ti in range(len(self.tenants)) if head[ti] < arrived[ti] and ti not in blocked]
                if not ready:
                    break
                ti = min(ready, key=lambda i: t_arr[i][head[i]])  # oldest waiting request first
                n = min(arrived[ti] - head[ti], max_batch, self.buckets[-1])
                adm = self._admit(ti, n)
                if adm is None:
                    blocked.add(ti)  # waits for a running batch to release its range
                    waits_mem += 1
                    continue
                bucket, off = adm
                n = min(n, bucket)
                self._launch(s, ti, order[ti][head[ti]: head[ti] + n], bucket, off)
                sizes.append(n)
                head[ti] += n
            if all(s.batch is None for s in self.slots) and all(
                    head[ti] >= arrived[ti] for ti in range(len(self.tenants))) and done < n_all:
                nxt = min(t_arr[ti][head[ti]] for ti in range(len(self.tenants)) if head[ti] < len(t_arr[ti]))
                wait = nxt - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.001))
        wall = time.perf_counter() - t0
        lat = (self._done - arr) * 1e3
        st = max(int(s.status.item()) for s in self.slots)
        summary = {"requests": n_all, "wall_s": wall, "qps": n_all / wall,
                   "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                   "mean_batch": float(np.mean(sizes)), "batches": len(sizes), "status": st,
                   "admission_waits": waits_mem, "graph_captures": self.captures,
                   "arena_bytes": self.arena.size}
        per = {}
        for ti in range(len(self.tenants)):
            m = ten == ti
            if m.any():
                per[ti] = {"requests": int(m.sum()), "p50_ms": float(np.percentile(lat[m], 50)),
                           "p99_ms": float(np.percentile(lat[m], 99))}
        summary["tenants"] = per
        return self._ids, self._dists, self._done, summary

    def serve_arrays(self, Q, K, nprobe, arrival, max_batch: int = 1024):
        """One tenant: request i is Q[i].  Returns (ids, dists, done, summary)."""
        n = len(Q)
        return self.serve_pool([Q], np.zeros(n, np.int64), np.arange(n), K, nprobe, arrival, max_batch)

    def serve(self, requests: list, max_batch: int = 1024) -> dict:
        """serve_pool() for Request objects: fills each request's ids, dists
        (its first K) and completion time."""
        pools = [[] for _ in self.tenants]
        qi = []
        for r in requests:
            qi.append(len(pools[r.tenant]))
            pools[r.tenant].append(np.asarray(r.query, np.float32))
        pools = [np.stack(p) if p else np.zeros((0, self.D[ti]), np.float32) for ti, p in enumerate(pools)]
        ids, d, done, out = self.serve_pool(pools, [r.tenant for r in requests], qi, [r.K for r in requests],
                                            [r.nprobe for r in requests], [r.arrival for r in requests], max_batch)
        for i, r in enumerate(requests):
            r.ids, r.dists, r.done = ids[i, :r.K].copy(), d[i, :r.K].copy(), float(done[i])
        return out


def poisson_arrivals(n: int, rate: float, seed: int = 6) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate (requests/s)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
