"""Autotuner for dade_search: picks the step width Delta_d, the first wave
size and nprobe that give the highest throughput at a recall target.

For every (Delta_d, first wave) it raises nprobe until recall@k against the
given ground truth reaches the target, times that configuration (CUDA
events, median of `reps` batches after `warmup`), and keeps the fastest.
The full-dimension scan (mode "full") is tuned the same way as a reference.
Results can be cached in a JSON file keyed by the index shape and the GPU.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np


def recall_at(ids: np.ndarray, gt: np.ndarray, k: int) -> float:
    hit = 0
    for b in range(len(gt)):
        hit += len(set(ids[b, :k].tolist()) & set(gt[b, :k].tolist()))
    return hit / (k * len(gt))


class Bench:
    """Device-resident batch for repeated dade_search calls.  estimator
    "learned" uses the index's tables; "res" the Gaussian-bound test with
    multiplier res_m."""

    def __init__(self, G, idx, Q, K: int, max_nprobe: int, deltas=(8, 16, 32), schedules=None,
                 estimator: str = "learned", res_m: float = 8.0):
        import torch
        self.G, self.idx, self.torch = G, idx, torch
        self.estimator, self.res_m = estimator, res_m
        dev = torch.device("cuda")
        self.B, self.K = len(Q), K
        self.q = torch.from_numpy(np.ascontiguousarray(Q, np.float32)).to(dev)
        self.k = torch.full((self.B,), K, dtype=torch.int32, device=dev)
        self.np = torch.zeros(self.B, dtype=torch.int32, device=dev)
        self.ids = torch.empty(self.B * K, dtype=torch.int64, device=dev)
        self.d = torch.empty(self.B * K, dtype=torch.float32, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.stats = torch.zeros((self.B, 4), dtype=torch.int64, device=dev)
        sched = ((1, 1),) + tuple(schedules if schedules is not None else SCHEDULES)
        ws = max(G.dade_search_workspace_size(idx, self.B, dd, K, max_nprobe, mode=m, first_wave=fw,
                                              wave_growth_log2=g, estimator=estimator)
                 for m in ("prune", "full") for dd in deltas for fw, g in sched)
        self.ws = torch.empty(ws, dtype=torch.uint8, device=dev)

    def run(self, nprobe, delta_d, mode, first_wave=1, stats=False, growth=0, final_test=False,
            scan_kernel="auto", queries_per_unit=0):
        self.np.fill_(nprobe)
        if stats:
            self.stats.zero_()
        self._search(nprobe, delta_d, mode, first_wave, stats, growth, final_test, scan_kernel, queries_per_unit)

    def _search(self, nprobe, delta_d, mode, first_wave, stats, growth, final_test, scan_kernel, queries_per_unit):
        self.G.dade_search(self.idx, self.q, self.k, self.np, delta_d, self.ids, self.d, max_K=self.K,
                           max_nprobe=nprobe, mode=mode, status=self.status, first_wave=first_wave,
                           stats=self.stats if stats else None, workspace=self.ws, wave_growth_log2=growth,
                           final_test=final_test, estimator=self.estimator, res_m=self.res_m,
                           scan_kernel=scan_kernel if mode == "prune" else "auto",
                           queries_per_unit=queries_per_unit)

    def result(self) -> np.ndarray:
        self.torch.cuda.synchronize()
        st = int(self.status.item())
        if st:
            raise RuntimeError(f"device status {st}")
        return self.ids.view(self.B, self.K).cpu().numpy()

    def capture(self, nprobe, delta_d, mode, first_wave=1, growth=0, final_test=False, scan_kernel="auto",
                queries_per_unit=0):
        """One search of this configuration captured in a CUDA graph (the
        per-query nprobe is set outside the graph, once)."""
        torch = self.torch
        self.run(nprobe, delta_d, mode, first_wave, growth=growth, final_test=final_test, scan_kernel=scan_kernel,
                 queries_per_unit=queries_per_unit)  # kernel attributes and module loads outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(g, stream=s):
            self._search(nprobe, delta_d, mode, first_wave, False, growth, final_test, scan_kernel,
                         queries_per_unit)
        torch.cuda.synchronize()
        return g

    def time(self, nprobe, delta_d, mode, steps, warmup, first_wave=1, growth=0, final_test=False,
             scan_kernel="auto", queries_per_unit=0, graph=False):
        """Returns (total ms, per-step ms list), CUDA events on the stream;
        graph=True replays one captured search per step."""
        torch = self.torch
        kw = dict(growth=growth, final_test=final_test, scan_kernel=scan_kernel, queries_per_unit=queries_per_unit)
        if graph:
            g = self.capture(nprobe, delta_d, mode, first_wave, **kw)
            step = g.replay
        else:
            self.np.fill_(nprobe)
            step = (lambda: self._search(nprobe, delta_d, mode, first_wave, False, growth, final_test, scan_kernel,
                                         queries_per_unit))
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for e0, e1 in evs:
            e0.record()
            step()
            e1.record()
        t1.record()
        torch.cuda.synchronize()
        return t0.elapsed_time(t1), [a.elapsed_time(b) for a, b in evs]


def cache_key(G, idx, K: int, target: float, mode: str) -> str:
    import torch
    info = G.dade_index_info_get(idx)
    sizes = G.dade_index_list_sizes(idx)
    h = hashlib.sha256(sizes.tobytes()).hexdigest()[:12]
    return (f"{torch.cuda.get_device_name()}|N{info['N']}|D{info['D']}|nl{info['nlist']}|dt{info['dtype']}"
            f"|{h}|K{K}|r{target}|{mode}")


SCHEDULES = ((1, 1), (4, 1), (8, 1), (8, 2), (4, 2), (2, 30), (4, 30), (8, 30), (16, 30))
# (scan kernel, queries per unit, final test) tried at the chosen schedule
KNOBS = (("auto", 0, False), ("auto", 0, True), ("tensor", 64, False), ("tensor", 32, False),
         ("cuda", 0, False), ("cuda", 8, False))


def autotune(bench: Bench, gt: np.ndarray, target: float = 0.95, k_recall: int = 10,
             deltas=(8, 16, 32), schedules=SCHEDULES,
             nprobes=(8, 16, 24, 32, 48, 64, 96, 128, 192, 256), reps: int = 5, warmup: int = 2,
             mode: str = "prune", knobs=KNOBS):
    """Returns (best configuration, every configuration tried).

    The smallest nprobe whose full-dimension scan reaches the target is found
    first (pruning can only lose recall); every (Delta_d, first wave, growth)
    schedule is then timed from that nprobe up to the first that reaches the
    target, and the kernel knobs (scan kernel, queries per work unit, final
    test) are timed at the fastest.  Mode "full" tunes the full-dimension
    scan's schedule the same way."""
    tried = []
    start = 0
    for i, npb in enumerate(nprobes):
        bench.run(npb, 0, "full", 1)
        if recall_at(bench.result(), gt, k_recall) >= target:
            start = i
            break
    else:
        start = len(nprobes) - 1
    dds = deltas if mode == "prune" else (0,)
    for dd in dds:
        for fw, g in schedules:
            for npb in nprobes[start:]:
                bench.run(npb, dd, mode, fw, growth=g)
                rec = recall_at(bench.result(), gt, k_recall)
                _, per = bench.time(npb, dd, mode, reps, warmup, fw, growth=g)
                tried.append(dict(mode=mode, delta_d=dd, first_wave=fw, growth=g, nprobe=npb, recall=rec,
                                  ms=float(np.median(per)), final_test=False, scan_kernel="auto",
                                  queries_per_unit=0))
                if rec >= target:
                    break
    ok = [t for t in tried if t["recall"] >= target]
    best = min(ok, key=lambda t: t["ms"]) if ok else max(tried, key=lambda t: t["recall"])
    if mode == "prune" and bench.estimator != "pq":
        # kernel knobs at the chosen configuration: which estimate-and-prune
        # kernel runs the later waves and how many queries share a staged
        # tile; the test on the completed distance.  None changes the
        # decisions (up to the kernels' rounding), so recall is re-measured
        # but the nprobe search is not repeated.
        b = best
        for kern, qpu, fin in knobs:
            if (kern, qpu, fin) == ("auto", 0, False):
                continue
            try:
                bench.run(b["nprobe"], b["delta_d"], mode, b["first_wave"], growth=b["growth"], final_test=fin,
                          scan_kernel=kern, queries_per_unit=qpu)
                rec = recall_at(bench.result(), gt, k_recall)
            except Exception:  # a knob the index or step width does not support
                continue
            _, per = bench.time(b["nprobe"], b["delta_d"], mode, reps, warmup, b["first_wave"], growth=b["growth"],
                                final_test=fin, scan_kernel=kern, queries_per_unit=qpu)
            t = dict(b, ms=float(np.median(per)), final_test=fin, scan_kernel=kern, queries_per_unit=qpu, recall=rec)
            tried.append(t)
            if rec >= min(target, b["recall"]) and t["ms"] < best["ms"]:
                best = t
    return best, tried


def autotune_cached(G, idx, bench: Bench, gt, cache_path: str | None = None, **kw):
    """autotune() with a JSON cache of the chosen configuration."""
    key = cache_key(G, idx, bench.K, kw.get("target", 0.95), kw.get("mode", "prune"))
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    if key in cache:
        return cache[key], []
    best, tried = autotune(bench, gt, **kw)
    if cache_path:
        cache[key] = best
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return best, tried
