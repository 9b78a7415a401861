#!/usr/bin/env python
"""Benchmark: queries/s at recall@10 >= 0.95 of the estimate-and-prune IVF
search (SIFT-shaped 1M x 128, nlist 4096, K 100) on one GB300, next to the
full-dimension FP32 IVF scan on the same GPU and the oracle on host cores.

One "step" is one dade_search over the whole 10,000-query batch (rotation,
centroid scan, top-nprobe, work units, every wave's estimate-and-prune scan
and top-K merge, output), with the batch and the index resident in HBM.
The index (1.0 GB of slabs and original vectors) is larger than L2 (129 MB).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun every rank runs its own replica of the workload on its GPU
(the search is replicated, not sharded); value = all ranks' queries / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TARGET_RECALL = 0.95
NPROBES = [8, 16, 24, 32, 48, 64, 96, 128, 192, 256]
DELTAS = [8, 16, 32]
SERVING_RATES = [200_000, 1_000_000, 3_000_000]
METRIC = "QPS at recall@10>=0.95 (estimate-and-prune IVF search, SIFT-shaped 1M x 128, nlist 4096, K 100)"
# --workload gist1m: the GIST-shaped set (1M x 960, strong spectral decay,
# 1,000 queries, BF16 slabs for the estimate, FP32 exact distances)
WORKLOAD_INFO = {
    "sift1m": dict(metric=METRIC, slabs="f32",
                   desc="sift1m-shaped: N={N}, D=128 integer [0,255], 256-comp mixture lambda~i^-0.8"),
    "gist1m": dict(metric="QPS at recall@10>=0.95 (estimate-and-prune IVF search, GIST-shaped 1M x 960, nlist 4096, "
                          "K 100, BF16 slabs)", slabs="bf16",
                   desc="gist1m-shaped: N={N}, D=960, 512-comp mixture lambda~i^-1.3"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=None, help="database size override (debug)")
    ap.add_argument("--queries", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-estimators", action="store_true",
                    help="skip the RES and ADS comparison lines")
    ap.add_argument("--cpu-sample-queries", type=int, default=1000)
    ap.add_argument("--workload", default="sift1m", choices=sorted(WORKLOAD_INFO) + ["vmf10m", "serving"],
                    help="sift1m (the benchmark line), gist1m, vmf10m (20,000 uneven requests on 10M x 96) or "
                         "serving (Poisson arrivals against two resident indices)")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="serving: seconds of arrivals per rate")
    ap.add_argument("--serve-budget-gb", type=float, default=16.0, help="serving: workspace arena size")
    ap.add_argument("--serve-graphs", action="store_true", help="serving: replay CUDA graphs per batch shape")
    ap.add_argument("--slabs", default=None, choices=["f32", "bf16", "fp8"],
                    help="slab precision (default: f32 for sift1m, bf16 for gist1m)")
    ap.add_argument("--profile", default=None,
                    help="NPROBE,DELTA_D[,FIRST_WAVE[,GROWTH]]: skip the sweep and baselines; run W + K steps of that "
                         "configuration inside the NVTX range 'dade_timed' (for ncu captures)")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while running (SM clock, reasons)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-i", str(gpu_index), "-lms", "50"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        self.marks = []

    def mark(self):
        self.marks.append(time.time())

    def wait_ready(self, timeout_s=5.0):
        """Block until nvidia-smi has written its first sample, so that the
        samples cover the timed region that follows."""
        t0 = time.time()
        while self.p and time.time() - t0 < timeout_s:
            self.f.flush()
            if os.path.getsize(self.f.name) > 0:
                return
            time.sleep(0.02)

    def stop(self):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append(parts)
            except ValueError:
                pass
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[4:8]) if v.lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- workload
def make_workload(n=None, nq=None, name="sift1m"):
    import synth
    X, Q, T, cfg = synth.workload(name, N=n, n_queries=nq)
    return X, Q, T, cfg


def ground_truth(X, Q, k=10, chunk=1024):
    """Exact top-k by brute force: torch GEMM-based shortlist of 64 on the GPU,
    then FP64 re-ranking of the shortlist on the host (plumbing for the
    recall metric, not the measured path)."""
    import torch
    dev = torch.device("cuda")
    Xt = torch.from_numpy(X).to(dev)
    xn = (Xt * Xt).sum(1)
    out = np.empty((len(Q), k), np.int64)
    for a in range(0, len(Q), chunk):
        q = torch.from_numpy(Q[a:a + chunk]).to(dev)
        d = xn[None, :] - 2.0 * (q @ Xt.T)
        cand = torch.topk(d, 64, dim=1, largest=False).indices.cpu().numpy()
        for i in range(cand.shape[0]):
            c = cand[i]
            dd = ((X[c].astype(np.float64) - Q[a + i].astype(np.float64)) ** 2).sum(1)
            o = np.lexsort((c, dd))[:k]
            out[a + i] = c[o]
        del d
    del Xt
    torch.cuda.empty_cache()
    return out


SCAN_SOURCES = {"tc_scan_kernel": ["scan_tc.cu", "tc_common.cuh", "scan.cuh", "scan_steps.cuh"],
                "wave_scan_kernel": ["scan.cu", "scan.cuh", "scan_steps.cuh"]}
PROFILE_OF = {"tc_scan_kernel": "tc_scan_sift1m.md", "wave_scan_kernel": "wave_scan_sift1m.md"}


def traffic_from_profiles(kernel, kernel_src_hash):
    """Per-launch DRAM bytes of the scan kernel from the committed ncu summary,
    if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", PROFILE_OF[kernel])
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"kernel source sha256: ([0-9a-f]{12})", txt)
    t = re.search(r"dram bytes per launch \(full-size equivalent\): ([0-9.e+]+)", txt)
    if not m or not t or m.group(1) != kernel_src_hash:
        return None
    return float(t.group(1))


def kernel_hash(kernel="tc_scan_kernel", root=ROOT):
    """sha256 of the scan kernel's sources with comments and blank lines
    removed (a comment edit does not make the recorded counters stale)."""
    h = hashlib.sha256()
    for f in SCAN_SOURCES[kernel]:
        src = open(os.path.join(root, "paper_2404_16322_gb300", "csrc", "kernels", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        lines = [ln.rstrip() for ln in src.splitlines() if ln.strip()]
        h.update("\n".join(lines).encode())
    return h.hexdigest()[:12]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- oracle arm
def time_oracle(oidx, m1, beta, nprobe, delta_d, K, steps, first_wave, growth, final_test):
    """Times the oracle (plain FP64 C loop, every host thread) on batches of
    queries, probing included; returns (threads, seconds per batch)."""
    from oracle import search
    threads = search.max_threads()
    search.set_threads(threads)
    times = []
    for q in steps:
        t0 = time.perf_counter()
        pr = oidx.probe(oidx.rotate_queries(q), nprobe)  # probing is part of the query
        search.search(oidx, q, pr, nprobe, K, delta_d, np.asarray(m1, np.float64), np.asarray(beta, np.float64),
                      first_wave=first_wave, growth=max(1, growth),
                      final_rel=search.FINAL_REL if final_test else np.inf)
        times.append(time.perf_counter() - t0)
    return threads, times


def oracle_on_library_index(G, idx, X, Q, mean, R, slabs, nprobe, delta_d, K, n_queries, first_wave, growth,
                            final_test, name):
    """The oracle on the same inputs as the GPU line: the library's index
    (rotation, centroids, bucket assignment, fitted tables) over the same
    rows, searched for the first n_queries of the same batch."""
    from oracle import search
    oidx = search.OracleIndex(X, mean, R, G.dade_index_centroids(idx).astype(np.float64),
                              G.dade_index_assignment(idx), dtype=slabs)
    m1, beta = G.dade_get_correction(idx, delta_d)
    q = Q[:n_queries]
    threads, times = time_oracle(oidx, m1, beta, nprobe, delta_d, K, [q], first_wave, growth, final_test)
    # one thread, on a tenth of the sample
    q1 = q[:max(1, len(q) // 10)]
    search.set_threads(1)
    t0 = time.perf_counter()
    pr = oidx.probe(oidx.rotate_queries(q1), nprobe)
    search.search(oidx, q1, pr, nprobe, K, delta_d, np.asarray(m1, np.float64), np.asarray(beta, np.float64),
                  first_wave=first_wave, growth=max(1, growth),
                  final_rel=search.FINAL_REL if final_test else np.inf)
    one_thread = len(q1) / (time.perf_counter() - t0)
    search.set_threads(threads)
    del oidx
    sample = (f"oracle FP64 C loop on the first {len(q)} of the {len(Q)} queries against the same "
              f"{len(X)}-vector {name}-shaped index as the GPU line (the library's rotation, centroids, "
              f"assignment and fitted tables; {slabs} slabs emulated), nprobe {nprobe}, K {K}, delta_d {delta_d}, "
              f"first wave {first_wave}, growth 2^{max(1, growth)}; probing included")
    return dict(value=len(q) / float(np.median(times)), unit="queries/s", cores=threads, kind="oracle",
                sample=sample, one_thread_value=one_thread, one_thread_queries=len(q1), cpu_model=cpu_model())


def cpu_model() -> str:
    """The host CPU's model name (from /proc/cpuinfo or lscpu), for the record."""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def blas_kmeans(Xr, nlist, iters, seed, sample_n):
    """Buckets for the reference arm's index, from the oracle-rotated rows:
    Lloyd k-means on a seeded sample (norm-expansion distances by BLAS),
    then every row to its nearest centroid (input preparation, not timed)."""
    rng = np.random.default_rng(seed)
    S = Xr[np.sort(rng.choice(len(Xr), min(sample_n, len(Xr)), replace=False))]
    C = S[rng.choice(len(S), nlist, replace=False)].copy()

    def nearest(A):
        out = np.empty(len(A), np.int64)
        cn = (C * C).sum(1)
        for a in range(0, len(A), 65536):
            blk = A[a:a + 65536]
            out[a:a + len(blk)] = np.argmin(cn[None, :] - 2.0 * (blk @ C.T), axis=1)
        return out

    for _ in range(iters):
        a = nearest(S)
        cnt = np.bincount(a, minlength=nlist)
        sums = np.zeros_like(C)
        np.add.at(sums, a, S)
        nz = cnt > 0
        C[nz] = sums[nz] / cnt[nz, None]
    return C, nearest(Xr).astype(np.int32)


def reference_arm(args):
    """The oracle as the reference arm: the same SIFT-shaped workload (the
    1M rows, nlist 4096, nprobe 64, K 100, Delta_d 16, first wave 4 and one
    later wave -- the GPU arm's tuned configuration), an index prepared on
    the host (the oracle's FP64 PCA, buckets by a BLAS k-means, tables by
    the oracle's replay and fit on 300 training queries), then steps of a
    bounded sample of 1,000 queries each, timed."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    from oracle import fit, pca, search
    t0 = time.perf_counter()
    X, Q, T, cfg = synth.workload("sift1m")
    nlist, K, nprobe, dd, fw, gw = cfg["nlist"], cfg["K"], 64, 16, 4, 30
    rng = np.random.default_rng(1)
    mu, R, _ = pca.train_rotation(X[np.sort(rng.choice(len(X), 200_000, replace=False))])
    Xr = pca.rotate(X, mu, R)
    C, a = blas_kmeans(Xr, nlist, 4, 1, 200_000)
    del Xr
    oidx = search.OracleIndex(X, mu, R, C, a, dtype="f32")
    Tq = T[:300]
    prt = oidx.probe(oidx.rotate_queries(Tq), nprobe)
    rows = search.collect(oidx, Tq, prt, nprobe, K, dd)
    S = search.n_steps(oidx.D, dd)
    top, _, _ = search.search(oidx, Tq, prt, nprobe, K, dd, *search.disabled_tables(S))
    P, tau, lab = fit.label_rows(rows, top, cap=500_000)
    m1, beta, _ = fit.fit_correction(P, tau, lab, oidx.D, dd)
    del rows, P
    n_q = 1000
    nsteps = args.steps + args.warmup
    batches = [Q[(s * n_q) % len(Q):(s * n_q) % len(Q) + n_q] for s in range(nsteps)]
    threads, times = time_oracle(oidx, m1, beta, nprobe, dd, K, batches, fw, gw, False)
    wall = time.perf_counter() - t0
    timed = times[args.warmup:] or times
    ms = 1000.0 * float(np.mean(timed))
    value = n_q / (ms / 1000.0)
    sample = (f"oracle FP64 C loop, {n_q} queries per step of the 10,000-query batch, against the full "
              f"{len(X)}-vector sift1m-shaped set (nlist {nlist}; the oracle's PCA, buckets by BLAS k-means on a "
              f"200k sample, tables fitted by the oracle on 300 training queries), nprobe {nprobe}, K {K}, "
              f"delta_d {dd}, first wave {fw}, growth 2^{gw}; probing included")
    cb = dict(value=value, unit="queries/s", cores=threads, kind="oracle", sample=sample, cpu_model=cpu_model())
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_INFO["sift1m"]["desc"].format(N=len(X)) + f"; {n_q} queries per step",
                       "nprobe": nprobe, "K": K, "delta_d": dd, "first_wave": fw, "wave_growth_log2": gw},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- uneven requests
UNEVEN_METRIC = ("QPS of 20,000 uneven requests in one call (estimate-and-prune IVF search, vMF-like 10M x 96, "
                 "nlist 4096, K in [1,100], nprobe in [8,256])")
UNEVEN_SCHEDULES = ((8, 30), (4, 30), (16, 30), (8, 2))
UNEVEN_BUDGETS = (0, 32 << 30, 96 << 30)  # candidate-buffer bound: the library default (8 GiB), 32, 96 GiB


def uneven_requests(args, G, torch, world, rank, local):
    """The large-N uneven-request line: one dade_search over all 20,000
    requests (per-request K uniform in [1, 100] and nprobe in [8, 256]) on
    the 10M x 96 vMF-like set, BF16 (or FP8) slabs, graph-captured; the wave
    schedule is the fastest of a few; the full-dimension scan of the same
    requests beside it; recall against brute force on a sample."""
    t_setup = time.perf_counter()
    slabs = args.slabs or "bf16"
    X, Q, T, cfg = make_workload(args.n, args.queries, "vmf10m")
    nlist = cfg["nlist"] if args.n is None else max(16, int(round(args.n / 2441)))
    mean, R, _ = G.dade_train_rotation(X, sample_n=min(len(X), 1_000_000), seed=1)
    idx = G.ivf_build(X, mean, R, nlist, kmeans_iters=10, seed=1, dtype=slabs)
    dd, maxK, maxP = 16, 100, min(256, nlist)
    G.dade_fit_correction(idx, T, maxK, min(64, nlist), dd, target_recall=0.995, seed=1)
    B = len(Q)
    rng = np.random.default_rng(10)
    Kv = rng.integers(1, maxK + 1, B).astype(np.int32)
    Nv = np.minimum(rng.integers(8, 257, B), maxP).astype(np.int32)
    n_gt = min(B, 1000)
    gt = ground_truth(X, Q[:n_gt], 10)
    dev = torch.device("cuda")
    q = torch.from_numpy(Q).to(dev)
    k = torch.from_numpy(Kv).to(dev)
    npb = torch.from_numpy(Nv).to(dev)
    ids = torch.empty(B * maxK, dtype=torch.int64, device=dev)
    dists = torch.empty(B * maxK, dtype=torch.float32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    stats = torch.zeros((B, 4), dtype=torch.int64, device=dev)
    ws = torch.empty(max(G.dade_search_workspace_size(idx, B, dd, maxK, maxP, mode=m, first_wave=fw,
                                                      wave_growth_log2=g, candidate_budget_bytes=cb)
                         for m in ("prune", "full") for fw, g in UNEVEN_SCHEDULES + ((1, 1),)
                         for cb in UNEVEN_BUDGETS),
                     dtype=torch.uint8, device=dev)
    budget = 0

    def search(mode, fw, g, with_stats=False):
        G.dade_search(idx, q, k, npb, dd if mode == "prune" else 0, ids, dists, max_K=maxK, max_nprobe=maxP,
                      mode=mode, first_wave=fw, wave_growth_log2=g, status=status, workspace=ws,
                      stats=stats if with_stats else None, candidate_budget_bytes=budget)

    def timed(mode, fw, g, steps, warmup):
        search(mode, fw, g)  # outside the capture: kernel attributes, module loads
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(graph, stream=s):
            search(mode, fw, g)
        for _ in range(warmup):
            graph.replay()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in evs:
            e0.record()
            graph.replay()
            e1.record()
        torch.cuda.synchronize()
        if int(status.item()):
            raise RuntimeError(f"device status {int(status.item())}")
        return [a.elapsed_time(b) for a, b in evs]

    def recall():
        got = ids.view(B, maxK)[:n_gt].cpu().numpy()
        m10 = Kv[:n_gt] >= 10
        r10 = float(np.mean([len(set(got[b, :10].tolist()) & set(gt[b].tolist())) / 10
                             for b in np.flatnonzero(m10)])) if m10.any() else None
        r1 = float(np.mean(got[:, 0] == gt[:, 0]))
        return r10, r1

    tried = []
    for cb in UNEVEN_BUDGETS:
        budget = cb
        for fw, g in UNEVEN_SCHEDULES:
            per = timed("prune", fw, g, 5, 2)
            tried.append(dict(first_wave=fw, growth=g, candidate_budget_bytes=cb, ms=float(np.median(per))))
    best = min(tried, key=lambda t: t["ms"])
    fw, g, budget = best["first_wave"], best["growth"], best["candidate_budget_bytes"]
    setup_s = time.perf_counter() - t_setup

    sampler = ClockSampler(local)
    sampler.wait_ready()
    per = timed("prune", fw, g, args.steps, args.warmup)
    clocks = sampler.stop()
    ms_step = float(np.mean(per))
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms_step], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    value = world * B / (ms_step / 1000.0)
    r10, r1 = recall()
    fper = timed("full", 1, 1, args.steps, args.warmup)
    full_qps = B / (float(np.mean(fper)) / 1000.0)
    fr10, fr1 = recall()

    G.dade_stage_timing(True, tensor_only=True)
    G.dade_stage_timing_read()
    for _ in range(args.steps):
        search("prune", fw, g)
    scan_ms, scan_launches, scan_bytes = G.dade_stage_timing_read()
    G.dade_stage_timing(False)
    per_launch_ms = scan_ms / max(1, scan_launches)
    per_launch_bytes = scan_bytes / max(1, scan_launches)
    peak, peak_kind = peaks()
    achieved = per_launch_bytes / (per_launch_ms / 1000.0) / 1e9 if per_launch_ms > 0 else 0.0

    stats.zero_()
    search("prune", fw, g, with_stats=True)
    torch.cuda.synchronize()
    st = stats.cpu().numpy()

    # end to end: requests (vectors, K, nprobe) from pinned host memory in,
    # results out, every step
    q_h, k_h, n_h = (torch.from_numpy(Q).pin_memory(), torch.from_numpy(Kv).pin_memory(),
                     torch.from_numpy(Nv).pin_memory())
    ids_h = torch.empty(B * maxK, dtype=torch.int64).pin_memory()
    d_h = torch.empty(B * maxK, dtype=torch.float32).pin_memory()

    def e2e_step():
        q.copy_(q_h, non_blocking=True)
        k.copy_(k_h, non_blocking=True)
        npb.copy_(n_h, non_blocking=True)
        search("prune", fw, g)
        ids_h.copy_(ids, non_blocking=True)
        d_h.copy_(dists, non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        e2e_step()
    e1.record()
    torch.cuda.synchronize()
    e2e_qps = world * B / (e0.elapsed_time(e1) / args.steps / 1000.0)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import search as osearch
        oidx = osearch.OracleIndex(X, mean, R, G.dade_index_centroids(idx).astype(np.float64),
                                   G.dade_index_assignment(idx), dtype=slabs)
        m1, beta = G.dade_get_correction(idx, dd)
        nq = min(B, max(20, args.cpu_sample_queries // 5))
        threads = osearch.max_threads()
        osearch.set_threads(threads)
        t0 = time.perf_counter()
        pr = oidx.probe(oidx.rotate_queries(Q[:nq]), maxP)
        osearch.search(oidx, Q[:nq], pr, Nv[:nq], Kv[:nq], dd, m1.astype(np.float64), beta.astype(np.float64),
                       first_wave=fw, growth=g)
        cpu_s = time.perf_counter() - t0
        del oidx
        cpu = dict(value=nq / cpu_s, unit="queries/s", cores=threads, kind="oracle", cpu_model=cpu_model(),
                   sample=f"oracle FP64 C loop on the first {nq} of the {B} requests (their own K and nprobe) "
                          f"against the same {len(X)}-vector index as the GPU line (the library's rotation, "
                          f"centroids, assignment and fitted table; {slabs} slabs emulated), delta_d {dd}, "
                          f"first wave {fw}, growth 2^{g}; probing included")

    line = {
        "metric": UNEVEN_METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"vmf10m-shaped: N={len(X)}, D=96, L2-normalised vMF mixture of 2048 components; "
                               f"B={B} requests, K~U[1,100], nprobe~U[8,256]; nlist={nlist}",
                   "delta_d": dd, "first_wave": fw, "wave_growth_log2": g, "slabs": slabs,
                   "candidate_budget_bytes": budget,
                   "recall@10(K>=10)": r10, "recall@1": r1, "graph": True, "parallelism": f"replicas x{world}",
                   "l2": f"inputs larger than L2 (index {G.dade_index_info_get(idx)['device_bytes'] / 1e9:.1f} GB "
                         "> 129 MB L2)",
                   "workspace_bytes": int(ws.numel())},
        "full_scan": {"value": full_qps, "unit": "queries/s", "recall@10(K>=10)": fr10, "recall@1": fr1},
        "speedup_vs_full_scan": value / world / full_qps,
        "scanned_dims_ratio": float(st[:, 3].sum() / max(1, st[:, 0].sum() * 96)),
        "latency_ms": {"batch_p50": float(np.percentile(per, 50)), "batch_p99": float(np.percentile(per, 99))},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind, "kernel": "tc_scan_kernel",
                     "per_launch_ms": per_launch_ms, "algorithmic_bytes_per_launch": per_launch_bytes,
                     "launches": scan_launches},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_qps, "unit": "queries/s", "h2d_bytes_per_step": int(Q.nbytes + Kv.nbytes + Nv.nbytes),
                "d2h_bytes_per_step": int(B * maxK * 12)},
        "gpu_launches": args.steps * G.dade_search_kernel_count(
            idx, q, k, npb, dd, ids, dists, max_K=maxK, max_nprobe=maxP, workspace=ws, status=status,
            first_wave=fw, wave_growth_log2=g, candidate_budget_bytes=budget),
        "clocks": clocks,
        "schedules": tried,
        "setup_s": setup_s,
    }
    idx.close()
    return line


# ---------------------------------------------------------------- two-index serving
SERVING_METRIC = ("serving QPS with p50/p99 latency (Poisson arrivals, two resident indices 2M x 256 and "
                  "1M x 960, BF16 slabs, K in {1,10,100}, nprobe in [8,512], memory-budget admission)")
SERVING5_RATES = [10_000, 20_000, 50_000, 100_000, 200_000]


def serving_two_indices(args, G, torch, world, rank, local):
    """Continuous batching against two resident indices (the serve2m-shaped
    2M x 256 set and the GIST-shaped 1M x 960 set, BF16 slabs): Poisson
    arrivals at each rate for --serve-seconds, every request for either
    index with equal probability, K uniform in {1, 10, 100} and nprobe
    uniform in [8, 512]; workspaces admitted from one arena of
    --serve-budget-gb.  Recall against brute force of the request's own
    query (recall@10 for K >= 10, recall@1 for K = 1)."""
    from paper_2404_16322_gb300 import serving
    t_setup = time.perf_counter()
    names = ("serve2m", "gist1m")
    tenants, pools, gts, info = [], [], [], []
    for name in names:
        X, Q, T, cfg = make_workload(args.n if name == "serve2m" else None, None, name)
        nq = min(len(Q), 2000)
        Q = Q[:nq]
        nlist = cfg["nlist"] if args.n is None else max(16, int(round(len(X) / 488)))
        mean, R, _ = G.dade_train_rotation(X, sample_n=min(len(X), 200_000), seed=1)
        idx = G.ivf_build(X, mean, R, nlist, kmeans_iters=10, seed=1, dtype="bf16")
        dd = 32
        G.dade_fit_correction(idx, T[:4000], 100, min(64, nlist), dd, target_recall=0.995, seed=1)
        tenants.append(serving.Tenant(idx, dd, 100, min(512, nlist), first_wave=8, wave_growth_log2=30))
        pools.append(Q)
        gts.append(ground_truth(X, Q, 10))
        info.append(f"{name}: N={len(X)}, D={X.shape[1]}, nlist={nlist}, {nq}-query pool")
        del X, T
    budget = int(args.serve_budget_gb * (1 << 30))
    srv = serving.Server(G, tenants, buckets=(16, 64, 256, 1024, 2048), slots=4, mem_budget=budget,
                         use_graphs=args.serve_graphs)
    # warm-up traffic (first use of each slot stream, pinned pages, arena offsets); not reported
    wn = 4000
    srv.serve_pool(pools, np.arange(wn) % 2, np.arange(wn) % min(len(p) for p in pools), np.full(wn, 10),
                   np.full(wn, 64), serving.poisson_arrivals(wn, 20_000, seed=5), max_batch=2048)
    setup_s = time.perf_counter() - t_setup
    rng = np.random.default_rng(6)
    out = []
    sampler = ClockSampler(local)
    sampler.wait_ready()
    for rate in SERVING5_RATES:
        n_req = int(rate * args.serve_seconds)
        arr = serving.poisson_arrivals(n_req, rate, seed=6)
        ten = rng.integers(0, 2, n_req)
        qi = rng.integers(0, min(len(p) for p in pools), n_req)
        ks = rng.choice([1, 10, 100], n_req)
        nps = np.minimum(rng.integers(8, 513, n_req), np.array([t.max_nprobe for t in tenants])[ten])
        ids, _, _, o = srv.serve_pool(pools, ten, qi, ks, nps, arr, max_batch=2048)
        r10, r1 = [], []
        for i in range(n_req):
            g = gts[ten[i]][qi[i]]
            if ks[i] >= 10:
                r10.append(len(set(ids[i, :10].tolist()) & set(g.tolist())) / 10)
            else:
                r1.append(float(ids[i, 0] == g[0]))
        o.update(offered_rate=rate, seconds=args.serve_seconds, recall_at_10=float(np.mean(r10)),
                 recall_at_1=float(np.mean(r1)))
        out.append(o)
    clocks = sampler.stop()
    ok = [o for o in out if o["status"] == 0 and o["qps"] >= 0.95 * o["offered_rate"]]
    best = max(ok, key=lambda o: o["offered_rate"]) if ok else max(out, key=lambda o: o["qps"])
    line = {
        "metric": SERVING_METRIC, "value": best["qps"], "unit": "queries/s", "n_gpus": world,
        "steps": len(out), "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "; ".join(info), "slabs": "bf16", "delta_d": 32, "first_wave": 8,
                   "wave_growth_log2": 30, "buckets": srv.buckets, "slots": len(srv.slots),
                   "arena_bytes": srv.arena.size, "graphs": args.serve_graphs,
                   "parallelism": f"replicas x{world}"},
        "p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"], "recall@10": best["recall_at_10"],
        "recall@1": best["recall_at_1"],
        "rates": out,
        "clocks": clocks,
        "setup_s": setup_s,
    }
    for t in tenants:
        t.idx.close()
    return line


# ---------------------------------------------------------------- main arm
def compare_estimators(G, X, Q, T, gt, idx, mean, R, nlist, K, slabs, maxp, nps, steps, warmup):
    """The other estimators of the paper on the same data and buckets, each
    autotuned to the same recall target and timed like the main line:
      res: the Gaussian-bound test of Section IV-C on the PCA index, m = 8
           (the paper's multiplier for SIFT- and GIST-like data);
      ads: ADS (Section III) -- a Haar-random rotation of the same buckets
           (centroids mapped through the rotations) and the scaled test with
           eps0 = 2.1, Delta_d = 32 (the paper's ADS setting);
      opq: OPQ-L (Section V-B) -- m = D/4 subspaces (D/8 for D = 960, the
           paper's settings) of 256 centroids on the same index, the
           three-feature classifier fitted on the training queries."""
    from paper_2404_16322_gb300 import autotune
    D = X.shape[1]
    esz = {"f32": 4, "bf16": 2, "fp8": 1}[slabs]
    out = {}

    def measure(run, best, per_candidate_bytes=0, exact_reads_slab=True):
        total, per = run.time(best["nprobe"], best["delta_d"], "prune", steps, warmup,
                              first_wave=best["first_wave"], growth=best["growth"], final_test=best["final_test"])
        run.run(best["nprobe"], best["delta_d"], "prune", stats=True, first_wave=best["first_wave"],
                growth=best["growth"], final_test=best["final_test"])
        run.result()
        st = run.stats.cpu().numpy()
        pruned_dims = st[:, 3] - st[:, 2] * D
        return {"value": run.B / (total / steps / 1000.0), "unit": "queries/s", "nprobe": best["nprobe"],
                "delta_d": best["delta_d"], "first_wave": best["first_wave"], "wave_growth_log2": best["growth"],
                "final_test": best["final_test"], "recall@10": best["recall"],
                "scanned_dims_ratio": float(st[:, 3].sum() / (st[:, 0].sum() * D)),
                "bytes_per_query": float((pruned_dims * esz + st[:, 2] * (D * esz * exact_reads_slab + D * 4)
                                          + st[:, 0] * per_candidate_bytes).sum() / run.B)}

    run = autotune.Bench(G, idx, Q, K, maxp, DELTAS, estimator="res", res_m=8.0)
    best, _ = autotune.autotune(run, gt, TARGET_RECALL, 10, DELTAS, nprobes=nps, mode="prune")
    out["res"] = dict(measure(run, best), res_m=8.0)
    del run

    Rh = G.dade_random_rotation(D, seed=4)
    C = G.dade_index_centroids(idx).astype(np.float64) @ R     # back to the centred input space
    Ch = (C @ Rh.T).astype(np.float32)
    ads_idx = G.ivf_build(X, mean, Rh, nlist, dtype=slabs, centroids=Ch, assign=G.dade_index_assignment(idx))
    m1, beta = G.dade_ads_table(D, 32, 2.1)
    G.dade_set_correction(ads_idx, 32, m1, beta)
    run = autotune.Bench(G, ads_idx, Q, K, maxp, (32,))
    best, _ = autotune.autotune(run, gt, TARGET_RECALL, 10, (32,), nprobes=nps, mode="prune")
    out["ads"] = dict(measure(run, best), eps0=2.1)
    del run
    ads_idx.close()

    m = D // 8 if D == 960 else D // 4
    t0 = time.perf_counter()
    rng = np.random.default_rng(7)
    sample = X[np.sort(rng.choice(len(X), min(len(X), 65536 if D <= 256 else 32768), replace=False))]
    G.dade_pq_train(idx, sample, m, iters=10, seed=1)
    G.dade_pq_fit_correction(idx, T, K, min(64, nlist), target_recall=0.995, seed=1)
    train_s = time.perf_counter() - t0
    run = autotune.Bench(G, idx, Q, K, maxp, (16,), estimator="pq")
    best, _ = autotune.autotune(run, gt, TARGET_RECALL, 10, (16,), nprobes=nps, mode="prune")
    out["opq"] = dict(measure(run, best, per_candidate_bytes=m, exact_reads_slab=False), m=m,
                      train_and_fit_s=train_s)
    del run
    return out


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2404_16322_gb300 as G
    from paper_2404_16322_gb300 import build as gbuild
    gbuild.build()

    if args.workload in ("vmf10m", "serving"):
        fn = uneven_requests if args.workload == "vmf10m" else serving_two_indices
        line = fn(args, G, torch, world, rank, local)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    t_setup = time.perf_counter()
    wl = WORKLOAD_INFO[args.workload]
    slabs = args.slabs or wl["slabs"]
    X, Q, T, cfg = make_workload(args.n, args.queries, args.workload)
    D = X.shape[1]
    K, nlist = cfg["K"], cfg["nlist"]
    if args.n is not None:
        nlist = max(16, int(round(args.n / 244)))
    mean, R, _ = G.dade_train_rotation(X, sample_n=min(len(X), 1_000_000 if D <= 256 else 200_000), seed=1)
    idx = G.ivf_build(X, mean, R, nlist, kmeans_iters=10, seed=1, dtype=slabs)
    fit_nprobe = min(64, nlist)
    fit_deltas = DELTAS if not args.profile else [int(args.profile.split(",")[1])]
    for dd in fit_deltas:
        G.dade_fit_correction(idx, T, K, fit_nprobe, dd, target_recall=0.995, seed=1)
    gt = ground_truth(X, Q, 10)
    setup_s = time.perf_counter() - t_setup

    from paper_2404_16322_gb300 import autotune, serving
    maxp = min(512 if args.workload == "gist1m" else max(NPROBES), nlist)
    run = autotune.Bench(G, idx, Q, K, maxp, DELTAS)
    if args.profile:
        vals = [int(x) for x in args.profile.split(",")]
        npb, dd = vals[0], vals[1]
        fw = vals[2] if len(vals) > 2 else 1
        gw = vals[3] if len(vals) > 3 else 1
        for _ in range(args.warmup):
            run.run(npb, dd, "prune", first_wave=fw, growth=gw)
        run.result()
        torch.cuda.nvtx.range_push("dade_timed")
        for _ in range(args.steps):
            run.run(npb, dd, "prune", first_wave=fw, growth=gw)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        ids = run.result()
        print(json.dumps({"profile": args.profile, "recall@10": autotune.recall_at(ids, gt, 10), "steps": args.steps,
                          "launches_per_step": G.dade_search_kernel_count(
                              idx, run.q, run.k, run.np, dd, run.ids, run.d, max_K=K, max_nprobe=npb,
                              workspace=run.ws, first_wave=fw, wave_growth_log2=gw), "setup_s": time.perf_counter() - t_setup}))
        return
    nps = [p for p in NPROBES + ([384, 512] if args.workload == "gist1m" else []) if p <= maxp]
    bd, tried_p = autotune.autotune(run, gt, TARGET_RECALL, 10, DELTAS, nprobes=nps, mode="prune")
    bf, tried_f = autotune.autotune(run, gt, TARGET_RECALL, 10, DELTAS, nprobes=nps, mode="full")
    sweep = tried_f + tried_p

    # --- timed region: exactly K steps of the chosen configuration
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.wait_ready()
    kn = dict(first_wave=bd["first_wave"], growth=bd["growth"], final_test=bd["final_test"],
              scan_kernel=bd.get("scan_kernel", "auto"), queries_per_unit=bd.get("queries_per_unit", 0))
    graph = run.capture(bd["nprobe"], bd["delta_d"], "prune", **kn)  # the timed step: one graph replay
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0e.record()
    for e0, e1 in evs:
        e0.record()
        graph.replay()
        e1.record()
    t1e.record()
    torch.cuda.synchronize()
    total_ms, per = t0e.elapsed_time(t1e), [a.elapsed_time(b) for a, b in evs]
    run.result()  # raises on a device status
    del graph
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_step = total_ms / args.steps
    value = world * run.B / (ms_step / 1000.0)

    # --- full-scan reference point on the same GPU, same timing
    f_total, f_per = run.time(bf["nprobe"], 0, "full", args.steps, args.warmup, first_wave=bf["first_wave"],
                              growth=bf["growth"], graph=True)
    full_qps = run.B / (f_total / args.steps / 1000.0)

    # --- stage timing of the dominant kernel (the estimate-and-prune scan of
    # the waves after the first: the tensor-core kernel unless the tuner
    # chose the CUDA-core one)
    tensor_scan = kn["scan_kernel"] != "cuda"
    G.dade_stage_timing(True, tensor_only=tensor_scan)
    G.dade_stage_timing_read()
    for _ in range(args.steps):
        run.run(bd["nprobe"], bd["delta_d"], "prune", **kn)
    scan_ms, scan_launches, scan_bytes = G.dade_stage_timing_read()
    G.dade_stage_timing(False)
    per_launch_ms = scan_ms / max(1, scan_launches)
    per_launch_bytes = scan_bytes / max(1, scan_launches)
    peak, peak_kind = peaks()
    achieved = per_launch_bytes / (per_launch_ms / 1000.0) / 1e9 if per_launch_ms > 0 else 0.0
    kname = "tc_scan_kernel" if tensor_scan else "wave_scan_kernel"
    khash = kernel_hash(kname)
    traffic = traffic_from_profiles(kname, khash) if args.workload == "sift1m" else None

    # --- work accounting (bytes per query) for both modes
    run.run(bd["nprobe"], bd["delta_d"], "prune", stats=True, **kn)
    run.result()
    st = run.stats.cpu().numpy()
    esz = {"f32": 4, "bf16": 2, "fp8": 1}[slabs]
    pruned_dims = st[:, 3] - st[:, 2] * D
    dade_bytes = (pruned_dims * esz + st[:, 2] * (D * esz + D * 4)).sum() / run.B
    run.run(bf["nprobe"], 0, "full", stats=True, first_wave=bf["first_wave"], growth=bf["growth"])
    run.result()
    stf = run.stats.cpu().numpy()
    full_bytes = (stf[:, 0] * D * 4).sum() / run.B
    scan_ratio = st[:, 3].sum() / (st[:, 0].sum() * D)

    # --- end to end through the C ABI with host buffers
    q_h = torch.from_numpy(Q).pin_memory()
    k_h = torch.full((run.B,), K, dtype=torch.int32).pin_memory()
    n_h = torch.full((run.B,), bd["nprobe"], dtype=torch.int32).pin_memory()
    ids_h = torch.empty(run.B * K, dtype=torch.int64).pin_memory()
    d_h = torch.empty(run.B * K, dtype=torch.float32).pin_memory()

    def e2e_step():
        run.q.copy_(q_h, non_blocking=True)
        run.k.copy_(k_h, non_blocking=True)
        run.np.copy_(n_h, non_blocking=True)
        G.dade_search(idx, run.q, run.k, run.np, bd["delta_d"], run.ids, run.d, max_K=K,
                      max_nprobe=bd["nprobe"], status=run.status, workspace=run.ws,
                      first_wave=bd["first_wave"], wave_growth_log2=bd["growth"], final_test=bd["final_test"],
                      scan_kernel=kn["scan_kernel"], queries_per_unit=kn["queries_per_unit"])
        ids_h.copy_(run.ids, non_blocking=True)
        d_h.copy_(run.d, non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        e2e_step()
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    e2e_qps = world * run.B / (e2e_ms / 1000.0)
    h2d = Q.nbytes + 2 * run.B * 4
    d2h = run.B * K * (8 + 4)
    assert np.array_equal(ids_h.view(run.B, K).numpy()[:, :10], run.result()[:, :10])

    # --- serving: Poisson arrivals of single-query requests (K in {1, 10, 100})
    serve_out = []
    if not args.no_serving:
        srv = serving.Server(G, idx, bd["delta_d"], max_K=K, max_nprobe=bd["nprobe"],
                             buckets=(64, 256, 1024, 4096), slots=3, first_wave=bd["first_wave"],
                             wave_growth_log2=bd["growth"], final_test=bd["final_test"])
        rng = np.random.default_rng(6)
        for rate in SERVING_RATES:
            n_req = int(min(200_000, max(20_000, rate * 0.25)))
            arr = serving.poisson_arrivals(n_req, rate, seed=6)
            ks = rng.choice([1, 10, 100], n_req)
            qi = np.arange(n_req) % len(Q)
            _, _, _, o = srv.serve_arrays(Q[qi], ks, np.full(n_req, bd["nprobe"]), arr, max_batch=4096)
            o["offered_rate"] = rate
            serve_out.append(o)
        del srv

    estimators = None
    if not args.no_estimators:
        estimators = compare_estimators(G, X, Q, T, gt, idx, mean, R, nlist, K, slabs, maxp, nps, args.steps,
                                        args.warmup)
        estimators["learned"] = {"value": value / world, "unit": "queries/s", "nprobe": bd["nprobe"],
                                 "delta_d": bd["delta_d"], "recall@10": bd["recall"], "scanned_dims_ratio": scan_ratio,
                                 "bytes_per_query": dade_bytes}
        estimators["speedup_learned_vs_ads"] = value / world / estimators["ads"]["value"]
        estimators["speedup_learned_vs_res"] = value / world / estimators["res"]["value"]
        estimators["speedup_learned_vs_opq"] = value / world / estimators["opq"]["value"]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_on_library_index(G, idx, X, Q, mean, R, slabs, bd["nprobe"], bd["delta_d"], K,
                                      args.cpu_sample_queries if D <= 256 else max(20, args.cpu_sample_queries // 5),
                                      bd["first_wave"], bd["growth"], bd["final_test"], args.workload)

    run.np.fill_(bd["nprobe"])
    launches = G.dade_search_kernel_count(idx, run.q, run.k, run.np, bd["delta_d"], run.ids, run.d, max_K=K,
                                          max_nprobe=bd["nprobe"], workspace=run.ws, status=run.status,
                                          first_wave=bd["first_wave"], wave_growth_log2=bd["growth"],
                                          final_test=bd["final_test"], scan_kernel=kn["scan_kernel"],
                                          queries_per_unit=kn["queries_per_unit"])
    line = {
        "metric": wl["metric"], "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["desc"].format(N=len(X)) + f"; B={run.B} queries; nlist={nlist}, K={K}",
                   "nprobe": bd["nprobe"], "delta_d": bd["delta_d"], "first_wave": bd["first_wave"],
                   "wave_growth_log2": bd["growth"], "final_test": bd["final_test"],
                   "scan_kernel": kn["scan_kernel"], "queries_per_unit": kn["queries_per_unit"], "graph": True,
                   "slabs": slabs, "recall@10": bd["recall"],
                   "parallelism": f"replicas x{world}",
                   "l2": f"inputs larger than L2 (index {G.dade_index_info_get(idx)['device_bytes'] / 1e9:.1f} GB > "
                         "129 MB L2)"},
        "full_scan": {"value": full_qps, "unit": "queries/s", "nprobe": bf["nprobe"], "recall@10": bf["recall"]},
        "speedup_vs_full_scan": value / world / full_qps,
        "bytes_per_query": {"prune": dade_bytes, "full_scan": full_bytes, "ratio": dade_bytes / full_bytes},
        "scanned_dims_ratio": scan_ratio,
        "latency_ms": {"batch_p50": float(np.percentile(per, 50)), "batch_p99": float(np.percentile(per, 99))},
        "serving": serve_out,
        "estimators": estimators,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "dram_achieved": (traffic / (per_launch_ms / 1000.0) / 1e9
                                       if traffic and per_launch_ms > 0 else None),
                     "dram_frac": (traffic / (per_launch_ms / 1000.0) / 1e9 / peak
                                   if traffic and per_launch_ms > 0 else None),
                     "kernel": kname, "kernel_src_sha256": khash, "per_launch_ms": per_launch_ms,
                     "algorithmic_bytes_per_launch": per_launch_bytes, "launches": scan_launches},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_qps, "unit": "queries/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches * args.steps,
        "clocks": clocks,
        "sweep": sweep,
        "setup_s": setup_s,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
