"""Continuous-batching search server over the C ABI.

Requests (one query vector, its K and nprobe) arrive over time.  The server
keeps the index, the per-batch workspaces and the result buffers resident on
the device and runs a single scheduling loop:

* a request that has arrived waits in a queue until a *slot* is free and the
  device-memory budget admits the batch it joins;
* a free slot takes up to ``max_batch`` waiting requests (as many as the
  budget's remaining workspace bytes allow), pads them to the smallest batch
  bucket that holds them with inactive queries (K = 0, nprobe = 0), copies
  them from pinned host memory, runs dade_search and copies the results back,
  all on the slot's own stream, so batches of different slots overlap on the
  device;
* finished slots hand their results back and free their bytes and slot.

With ``use_graphs`` every (slot, bucket) pair is captured once as a CUDA graph
(host-to-device copies, the search, device-to-host copies) and replayed.

A query's result does not depend on the batch it travels in: the search's
wave schedule freezes each query's threshold per wave of its own probe ranks,
and every (query, candidate) distance is computed with the same arithmetic
whatever the batch.
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
    done: float = -1.0
    ids: np.ndarray | None = None
    dists: np.ndarray | None = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class _Slot:
    def __init__(self, torch, G, idx, D, bucket_sizes, max_K, max_nprobe, delta_d, mode, first_wave, ws_bytes,
                 growth=0, final_test=False):
        dev = torch.device("cuda")
        self.stream = torch.cuda.Stream()
        B = max(bucket_sizes)
        self.q_h = torch.zeros((B, D), dtype=torch.float32).pin_memory()
        self.k_h = torch.zeros(B, dtype=torch.int32).pin_memory()
        self.n_h = torch.zeros(B, dtype=torch.int32).pin_memory()
        self.ids_h = torch.empty(B * max_K, dtype=torch.int64).pin_memory()
        self.d_h = torch.empty(B * max_K, dtype=torch.float32).pin_memory()
        self.q = torch.zeros((B, D), dtype=torch.float32, device=dev)
        self.k = torch.zeros(B, dtype=torch.int32, device=dev)
        self.n = torch.zeros(B, dtype=torch.int32, device=dev)
        self.ids = torch.empty(B * max_K, dtype=torch.int64, device=dev)
        self.d = torch.empty(B * max_K, dtype=torch.float32, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        self.event = torch.cuda.Event()
        self.graphs = {}
        self.batch = None
        self.bucket = 0
        self.bytes = 0
        self.args = (G, idx, max_K, max_nprobe, delta_d, mode, first_wave, growth, final_test)

    def enqueue(self, torch, b: int):
        """H2D copies, the search over the first b rows, D2H copies."""
        G, idx, max_K, max_nprobe, delta_d, mode, first_wave, growth, final_test = self.args
        self.q[:b].copy_(self.q_h[:b], non_blocking=True)
        self.k[:b].copy_(self.k_h[:b], non_blocking=True)
        self.n[:b].copy_(self.n_h[:b], non_blocking=True)
        G.dade_search(idx, self.q[:b], self.k[:b], self.n[:b], delta_d, self.ids, self.d, max_K=max_K,
                      max_nprobe=max_nprobe, mode=mode, first_wave=first_wave, status=self.status,
                      workspace=self.ws, stream=torch.cuda.current_stream(), wave_growth_log2=growth,
                      final_test=final_test)
        self.ids_h[: b * max_K].copy_(self.ids[: b * max_K], non_blocking=True)
        self.d_h[: b * max_K].copy_(self.d[: b * max_K], non_blocking=True)


class Server:
    def __init__(self, G, idx, delta_d: int, max_K: int, max_nprobe: int, buckets=(16, 64, 256, 1024),
                 slots: int = 2, mem_budget: int | None = None, use_graphs: bool = True,
                 mode: str = "prune", first_wave: int = 1, wave_growth_log2: int = 0, final_test: bool = False):
        import torch
        self.torch, self.G, self.idx = torch, G, idx
        info = G.dade_index_info_get(idx)
        self.D = info["D"]
        self.max_K, self.max_nprobe = max_K, max_nprobe
        self.buckets = sorted(buckets)
        self.ws_of = {b: G.dade_search_workspace_size(idx, b, delta_d, max_K, max_nprobe, mode=mode,
                                                      first_wave=first_wave, wave_growth_log2=wave_growth_log2)
                      for b in self.buckets}
        ws_max = max(self.ws_of.values())
        self.mem_budget = mem_budget if mem_budget is not None else slots * ws_max
        if self.mem_budget < self.ws_of[self.buckets[0]]:
            raise ValueError("memory budget below the smallest batch's workspace")
        self.slots = [_Slot(torch, G, idx, self.D, self.buckets, max_K, max_nprobe, delta_d, mode, first_wave,
                            ws_max, wave_growth_log2, final_test) for _ in range(slots)]
        self.use_graphs = use_graphs
        # warm up every (slot, bucket): first launches configure kernels; then capture
        for s in self.slots:
            for b in self.buckets:
                s.k_h[:b] = 0
                s.n_h[:b] = 0
                with torch.cuda.stream(s.stream):
                    s.enqueue(torch, b)
                s.stream.synchronize()
                if use_graphs:
                    g = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(g, stream=s.stream):
                        s.enqueue(torch, b)
                    s.graphs[b] = g
        torch.cuda.synchronize()
        self.in_flight_bytes = 0

    def _bucket_for(self, n: int) -> int:
        for b in self.buckets:
            if b >= n:
                return b
        return self.buckets[-1]

    def _launch(self, s: _Slot, lo: int, hi: int, bucket: int):
        n = hi - lo
        s.q_h.numpy()[:n] = self._Q[lo:hi]
        s.k_h.numpy()[:n] = self._K[lo:hi]
        s.n_h.numpy()[:n] = self._NP[lo:hi]
        if bucket > n:
            s.k_h.numpy()[n:bucket] = 0
            s.n_h.numpy()[n:bucket] = 0
        torch = self.torch
        with torch.cuda.stream(s.stream):
            if self.use_graphs:
                s.graphs[bucket].replay()
            else:
                s.enqueue(torch, bucket)
            s.event.record(s.stream)
        s.batch, s.bucket, s.bytes = (lo, hi), bucket, self.ws_of[bucket]
        self.in_flight_bytes += s.bytes

    def _finish(self, s: _Slot, now: float):
        lo, hi = s.batch
        n, K = hi - lo, self.max_K
        self._ids[lo:hi] = s.ids_h.numpy()[: n * K].reshape(n, K)
        self._dists[lo:hi] = s.d_h.numpy()[: n * K].reshape(n, K)
        self._done[lo:hi] = now
        self.in_flight_bytes -= s.bytes
        s.batch = None

    def serve_arrays(self, Q, K, nprobe, arrival, max_batch: int = 1024):
        """Serve len(Q) requests given as arrays, in arrival order.  Returns
        (ids [n, max_K], dists [n, max_K], done times [n], summary)."""
        order = np.argsort(np.asarray(arrival, dtype=np.float64), kind="stable")
        self._Q = np.ascontiguousarray(np.asarray(Q, np.float32)[order])
        self._K = np.asarray(K, np.int32)[order]
        self._NP = np.asarray(nprobe, np.int32)[order]
        arr = np.asarray(arrival, np.float64)[order]
        n_all = len(arr)
        self._ids = np.full((n_all, self.max_K), -1, np.int64)
        self._dists = np.full((n_all, self.max_K), np.inf, np.float32)
        self._done = np.full(n_all, -1.0)
        head = 0      # first request not yet admitted (requests are FIFO by arrival)
        done = 0
        sizes = []
        t0 = time.perf_counter()
        while done < n_all:
            now = time.perf_counter() - t0
            arrived = int(np.searchsorted(arr, now, side="right"))
            for s in self.slots:
                if s.batch is not None and s.event.query():
                    done += s.batch[1] - s.batch[0]
                    self._finish(s, time.perf_counter() - t0)
            for s in self.slots:
                if s.batch is not None or head >= arrived:
                    continue
                n = min(arrived - head, max_batch, self.buckets[-1])
                bucket = self._bucket_for(n)
                # admission by memory: shrink the batch until its workspace fits
                while bucket > self.buckets[0] and self.in_flight_bytes + self.ws_of[bucket] > self.mem_budget:
                    bucket = self.buckets[self.buckets.index(bucket) - 1]
                if self.in_flight_bytes + self.ws_of[bucket] > self.mem_budget:
                    break
                n = min(n, bucket)
                self._launch(s, head, head + n, bucket)
                sizes.append(n)
                head += n
            if head >= arrived and head < n_all and all(s.batch is None for s in self.slots):
                wait = arr[head] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.001))
        wall = time.perf_counter() - t0
        lat = (self._done - arr) * 1e3
        st = max(int(s.status.item()) for s in self.slots)
        inv = np.empty_like(order)
        inv[order] = np.arange(n_all)
        summary = {"requests": n_all, "wall_s": wall, "qps": n_all / wall,
                   "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                   "mean_batch": float(np.mean(sizes)), "batches": len(sizes), "status": st}
        return self._ids[inv], self._dists[inv], self._done[inv], summary

    def serve(self, requests: list, max_batch: int = 1024) -> dict:
        """serve_arrays() for Request objects: fills each request's ids,
        dists (its first K) and completion time."""
        ids, d, done, out = self.serve_arrays([r.query for r in requests], [r.K for r in requests],
                                              [r.nprobe for r in requests], [r.arrival for r in requests],
                                              max_batch)
        for i, r in enumerate(requests):
            r.ids, r.dists, r.done = ids[i, :r.K].copy(), d[i, :r.K].copy(), float(done[i])
        return out


def poisson_arrivals(n: int, rate: float, seed: int = 6) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate (requests/s)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
