"""GB300 data-aware distance estimation for IVF refinement (arXiv 2404.16322).

A thin binding over the C ABI of ``include/dade.h``: every function below
has the C entry point's name and only marshals arguments (NumPy arrays for
host buffers, torch CUDA tensors for device buffers and streams).  Every step
of the search runs in the library's CUDA kernels; if the library is not
built, the first call raises.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L

__all__ = ["dade_train_rotation", "dade_random_rotation", "dade_ads_table", "ivf_build", "dade_fit_correction", "dade_fit_collect", "dade_fit_samples",
           "dade_set_correction", "dade_get_correction", "dade_search", "dade_search_noalloc",
           "dade_search_workspace_size",
           "dade_index_info_get", "dade_index_centroids", "dade_index_assignment",
           "dade_index_list_sizes", "dade_index_stored", "dade_index_save", "dade_index_load", "dade_index_free",
           "dade_stage_timing", "dade_stage_timing_read", "dade_last_error", "Index", "library",
           "n_steps", "dade_shard_owners", "dade_index_shard", "dade_merge_topk", "dade_pq_train", "dade_pq_set",
           "dade_pq_fit_correction", "dade_pq_fit_samples", "dade_pq_set_correction", "dade_pq_get"]

_LIB = None


def library() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = L.load()
    return _LIB


def dade_last_error() -> str:
    return library().dade_last_error().decode()


def _check(st: int) -> None:
    if st != 0:
        raise L.DadeError(st, dade_last_error())


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def n_steps(D: int, delta_d: int) -> int:
    return -(-(-(-D // 8) * 8) // delta_d)


class Index:
    """Owner of a ``dade_index*``; released by ``dade_index_free`` on close/del."""

    def __init__(self, handle: int):
        self.handle = ctypes.c_void_p(handle)

    @property
    def ptr(self):
        if not self.handle:
            raise ValueError("index is closed")
        return self.handle

    def close(self):
        if self.handle:
            library().dade_index_free(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover - interpreter shutdown
            pass

    def info(self) -> dict:
        return dade_index_info_get(self)


def dade_train_rotation(X, sample_n: int = 0, seed: int = 0):
    """PCA rotation on the host in FP64: returns (mean[D], R[D, D], eigvals[D])."""
    X = _host(X, np.float32)
    n, D = X.shape
    mean = np.empty(D)
    R = np.empty((D, D))
    lam = np.empty(D)
    _check(library().dade_train_rotation(X.ctypes.data, n, D, int(sample_n), int(seed), mean.ctypes.data,
                                         R.ctypes.data, lam.ctypes.data))
    return mean, R, lam


def dade_random_rotation(D: int, seed: int = 0):
    """Haar-random orthogonal R[D, D] (FP64, host): the ADS rotation."""
    R = np.empty((int(D), int(D)))
    _check(library().dade_random_rotation(int(D), int(seed), R.ctypes.data))
    return R


def dade_ads_table(D: int, delta_d: int, eps0: float = 2.1):
    """The correction table that makes the search's test ADS's
    (D/d) dis' > (1 + eps0/sqrt(d)) tau: returns (m1, beta), S - 1 floats."""
    S = n_steps(D, delta_d)
    m1 = np.zeros(max(S - 1, 1), np.float32)
    beta = np.zeros(max(S - 1, 1), np.float32)
    _check(library().dade_ads_table(int(D), int(delta_d), float(eps0), m1.ctypes.data, beta.ctypes.data))
    return m1[:S - 1], beta[:S - 1]


def ivf_build(X, mean, R, nlist: int, kmeans_iters: int = 10, seed: int = 0, dtype: str = "f32",
              centroids=None, assign=None, ids=None) -> Index:
    """X: (N, D) float32 rows, a NumPy array (host) or a contiguous CUDA
    tensor on the current device (read in place)."""
    if not isinstance(X, np.ndarray) and hasattr(X, "is_cuda") and X.is_cuda:
        import torch
        assert X.dtype == torch.float32 and X.is_contiguous() and X.dim() == 2
        xp = X.data_ptr()
    else:
        X = _host(X, np.float32)
        xp = X.ctypes.data
    N, D = X.shape
    mean = _host(mean, np.float64)
    R = _host(R, np.float64)
    c = None if centroids is None else _host(centroids, np.float32)
    a = None if assign is None else _host(assign, np.int32)
    i = None if ids is None else _host(ids, np.int64)
    p = L.BuildParams(int(nlist), int(kmeans_iters), int(seed), L.SLAB[dtype], _ptr(c), _ptr(a), _ptr(i))
    out = ctypes.c_void_p()
    _check(library().ivf_build(xp, N, D, mean.ctypes.data, R.ctypes.data, ctypes.byref(p),
                               ctypes.byref(out)))
    return Index(out.value)


def dade_fit_correction(idx: Index, T, K: int, nprobe: int, delta_d: int, target_recall: float = 0.995,
                        seed: int = 0, label1_cap: int = 500_000):
    T = _host(T, np.float32)
    info = dade_index_info_get(idx)
    S = n_steps(info["D"], delta_d)
    m1 = np.zeros(max(S - 1, 1), np.float32)
    beta = np.zeros(max(S - 1, 1), np.float32)
    _check(library().dade_fit_correction(idx.ptr, T.ctypes.data, T.shape[0], int(K), int(nprobe),
                                         int(delta_d), float(target_recall), int(seed), int(label1_cap),
                                         m1.ctypes.data, beta.ctypes.data))
    return m1[:S - 1], beta[:S - 1]


def dade_fit_collect(idx: Index, T, K: int, nprobe: int, delta_d: int, seed: int = 0, label1_cap: int = 500_000,
                     max_rows: int | None = None) -> dict:
    """The samples dade_fit_correction fits on, sorted by (query, id):
    dict(partials[n, S-1], tau[n], label[n], query[n], id[n])."""
    T = _host(T, np.float32)
    S = n_steps(dade_index_info_get(idx)["D"], delta_d)
    cap = int(max_rows) if max_rows is not None else len(T) * int(K) + int(label1_cap) + 4096
    n = ctypes.c_int64(0)
    P = np.empty((cap, max(S - 1, 1)), np.float32)
    tau = np.empty(cap, np.float32)
    lab = np.empty(cap, np.int8)
    qi = np.empty(cap, np.int64)
    ii = np.empty(cap, np.int64)
    _check(library().dade_fit_collect(idx.ptr, T.ctypes.data, len(T), int(K), int(nprobe), int(delta_d), int(seed),
                                      int(label1_cap), cap, ctypes.byref(n), P.ctypes.data, tau.ctypes.data,
                                      lab.ctypes.data, qi.ctypes.data, ii.ctypes.data))
    m = n.value
    return dict(partials=P[:m, :S - 1], tau=tau[:m], label=lab[:m], query=qi[:m], id=ii[:m])


def dade_partials_collect(idx: Index, Q, nprobe: int, delta_d: int, max_rows: int | None = None) -> dict:
    """Every candidate of each query's nprobe nearest buckets with its
    partial distances over the stored slabs, sorted by (query, id):
    dict(partials[n, S-1], query[n], id[n])."""
    Q = _host(Q, np.float32)
    info = dade_index_info_get(idx)
    S = n_steps(info["D"], delta_d)
    cap = int(max_rows) if max_rows is not None else len(Q) * int(info["N"])
    n = ctypes.c_int64(0)
    P = np.empty((max(cap, 1), max(S - 1, 1)), np.float32)
    qi = np.empty(max(cap, 1), np.int64)
    ii = np.empty(max(cap, 1), np.int64)
    _check(library().dade_partials_collect(idx.ptr, Q.ctypes.data, len(Q), int(nprobe), int(delta_d), cap,
                                           ctypes.byref(n), P.ctypes.data, qi.ctypes.data, ii.ctypes.data))
    m = n.value
    return dict(partials=P[:m, :S - 1], query=qi[:m], id=ii[:m])


class Arena:
    """Offsets into one caller-held device allocation of `size` bytes: the
    serving loop's admission control (first fit, aligned, coalescing)."""

    def __init__(self, size: int, align: int = 256):
        self.ptr = ctypes.c_void_p()
        _check(library().dade_arena_create(int(size), int(align), ctypes.byref(self.ptr)))
        self.size = int(size) // int(align) * int(align)

    def alloc(self, nbytes: int) -> int:
        """Offset of the range, or -1 when no free range holds nbytes."""
        return int(library().dade_arena_alloc(self.ptr, int(nbytes)))

    def free(self, offset: int) -> None:
        _check(library().dade_arena_free(self.ptr, int(offset)))

    @property
    def used(self) -> int:
        return int(library().dade_arena_used(self.ptr))

    @property
    def largest_free(self) -> int:
        return int(library().dade_arena_largest_free(self.ptr))

    def close(self):
        if self.ptr:
            library().dade_arena_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dade_fit_samples(partials, tau, label, D: int, delta_d: int, target_recall: float = 0.995,
                     min_label0: int = 100):
    P = _host(partials, np.float64)
    t = _host(tau, np.float64)
    lab = _host(label, np.int8)
    S = n_steps(D, delta_d)
    m1 = np.zeros(max(S - 1, 1))
    beta = np.zeros(max(S - 1, 1))
    _check(library().dade_fit_samples(P.ctypes.data, t.ctypes.data, lab.ctypes.data, len(t), int(D),
                                      int(delta_d), float(target_recall), int(min_label0), m1.ctypes.data,
                                      beta.ctypes.data))
    return m1[:S - 1], beta[:S - 1]


def dade_pq_train(idx: Index, X, m: int, iters: int = 10, seed: int = 0):
    """OPQ-L quantiser (parametric OPQ on the index's PCA basis, m subspaces
    of 256 centroids) trained on the rows of X (host FP32, original space);
    every stored vector is encoded on the device.  Returns (perm, codebooks)."""
    X = _host(X, np.float32)
    n, D = X.shape
    perm = np.empty(D, np.int32)
    cb = np.empty((int(m), 256, D // int(m)), np.float32)
    _check(library().dade_pq_train(idx.ptr, X.ctypes.data, n, int(m), int(iters), int(seed), perm.ctypes.data,
                                   cb.ctypes.data))
    return perm, cb


def dade_pq_set(idx: Index, perm, codebooks) -> None:
    perm = _host(perm, np.int32)
    cb = _host(codebooks, np.float32)
    _check(library().dade_pq_set(idx.ptr, int(cb.shape[0]), perm.ctypes.data, cb.ctypes.data))


def dade_pq_fit_correction(idx: Index, T, K: int, nprobe: int, target_recall: float = 0.995, seed: int = 0,
                           label1_cap: int = 500_000):
    """OPQ-L's three-feature classifier fitted on replayed training queries;
    returns (m1, m3, beta)."""
    T = _host(T, np.float32)
    out = np.zeros(3, np.float32)
    _check(library().dade_pq_fit_correction(idx.ptr, T.ctypes.data, len(T), int(K), int(nprobe), float(target_recall),
                                            int(seed), int(label1_cap), out.ctypes.data))
    return tuple(float(v) for v in out)


def dade_pq_fit_samples(dis, err, tau, label, target_recall: float = 0.995, min_label0: int = 100):
    d = _host(dis, np.float64)
    e = _host(err, np.float64)
    t = _host(tau, np.float64)
    lab = _host(label, np.int8)
    out = np.zeros(3)
    _check(library().dade_pq_fit_samples(d.ctypes.data, e.ctypes.data, t.ctypes.data, lab.ctypes.data, len(t),
                                         float(target_recall), int(min_label0), out.ctypes.data))
    return tuple(float(v) for v in out)


def dade_pq_set_correction(idx: Index, m1: float, m3: float, beta: float) -> None:
    _check(library().dade_pq_set_correction(idx.ptr, float(m1), float(m3), float(beta)))


def dade_pq_get(idx: Index, codes: bool = False):
    """(m, (m1, m3, beta) or None, codes[N, m] and err[N] in input-row order if asked)."""
    m = ctypes.c_int32(0)
    _check(library().dade_pq_get(idx.ptr, ctypes.byref(m), None, None, None))
    corr = np.zeros(3, np.float32)
    try:
        _check(library().dade_pq_get(idx.ptr, None, corr.ctypes.data, None, None))
        c3 = tuple(float(v) for v in corr)
    except L.DadeError:
        c3 = None
    if not codes:
        return m.value, c3
    N = dade_index_info_get(idx)["N"]
    cd = np.empty((N, m.value), np.uint8)
    er = np.empty(N, np.float32)
    _check(library().dade_pq_get(idx.ptr, None, None, cd.ctypes.data, er.ctypes.data))
    return m.value, c3, cd, er


def dade_set_correction(idx: Index, delta_d: int, m1, beta) -> None:
    m1 = _host(m1, np.float32)
    beta = _host(beta, np.float32)
    _check(library().dade_set_correction(idx.ptr, int(delta_d), m1.ctypes.data, beta.ctypes.data))


def dade_get_correction(idx: Index, delta_d: int):
    info = dade_index_info_get(idx)
    S = n_steps(info["D"], delta_d)
    m1 = np.zeros(max(S - 1, 1), np.float32)
    beta = np.zeros(max(S - 1, 1), np.float32)
    _check(library().dade_get_correction(idx.ptr, int(delta_d), m1.ctypes.data, beta.ctypes.data))
    return m1[:S - 1], beta[:S - 1]


def _opts(mode, max_K, max_nprobe, first_wave=0, tau=None, probe_in=None, probe_out=None, qrot_out=None,
          stats=None, status=None, workspace=None, wave_growth_log2=0, final_test=False, estimator="learned",
          res_m=8.0, test_steps=0, scan_kernel="auto", candidate_budget_bytes=0, queries_per_unit=0):
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    return L.SearchOpts(L.MODE[mode], int(max_K), int(max_nprobe), int(first_wave), _ptr(tau),
                        _ptr(probe_in), _ptr(probe_out), _ptr(qrot_out), _ptr(stats), _ptr(status),
                        _ptr(workspace), ws_bytes, int(wave_growth_log2), int(bool(final_test)),
                        L.ESTIMATOR[estimator], float(res_m), int(test_steps), L.SCAN_KERNEL[scan_kernel],
                        int(candidate_budget_bytes), int(queries_per_unit))


def dade_search_workspace_size(idx: Index, B: int, delta_d: int, max_K: int, max_nprobe: int,
                               mode: str = "prune", first_wave: int = 0, frozen: bool = False,
                               probe_in: bool = False, wave_growth_log2: int = 0, final_test: bool = False,
                               estimator: str = "learned", scan_kernel: str = "auto",
                               candidate_budget_bytes: int = 0, queries_per_unit: int = 0) -> int:
    o = _opts(mode, max_K, max_nprobe, first_wave, wave_growth_log2=wave_growth_log2, final_test=final_test,
              estimator=estimator, scan_kernel=scan_kernel, candidate_budget_bytes=candidate_budget_bytes,
              queries_per_unit=queries_per_unit)
    if frozen:
        o.tau_dev = 1  # only its presence matters for sizing
    if probe_in:
        o.probe_in_dev = 1
    return int(library().dade_search_workspace_size(idx.ptr, int(B), int(delta_d), ctypes.byref(o)))


def dade_search(idx: Index, Q, K, nprobe, delta_d: int, ids, dists, *, max_K: int, max_nprobe: int,
                mode: str = "prune", first_wave: int = 0, tau=None, probe_in=None, probe_out=None,
                qrot_out=None, stats=None, status=None, workspace=None, offsets=None, stream=None,
                wave_growth_log2: int = 0, final_test: bool = False, estimator: str = "learned",
                res_m: float = 8.0, test_steps: int = 0, scan_kernel: str = "auto",
                candidate_budget_bytes: int = 0, queries_per_unit: int = 0) -> None:
    """Enqueue a search on ``stream`` (a torch.cuda.Stream; default: current).

    Q: (B, D) float32 CUDA tensor; K, nprobe: (B,) int32 CUDA tensors; ids
    (int64) and dists (float32) are output CUDA tensors of B * max_K (or
    offsets[-1]) elements.  Optional tensors as in dade_search_opts;
    estimator "learned" (the installed tables) or "res" (the Gaussian-bound
    test with multiplier res_m); test_steps > 0 tests only the first
    test_steps steps; scan_kernel "auto" / "tensor" / "cuda" picks the
    estimate-and-prune kernel of the learned test; candidate_budget_bytes
    bounds the candidate buffer (0: the library default) and
    queries_per_unit the queries sharing one staged tile (0: the kernel's
    maximum)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    o = _opts(mode, max_K, max_nprobe, first_wave, tau, probe_in, probe_out, qrot_out, stats, status,
              workspace, wave_growth_log2, final_test, estimator, res_m, test_steps, scan_kernel,
              candidate_budget_bytes, queries_per_unit)
    _check(library().dade_search(idx.ptr, _ptr(Q), int(Q.shape[0]), _ptr(K), _ptr(nprobe), int(delta_d),
                                 ctypes.byref(o), _ptr(ids), _ptr(dists), _ptr(offsets),
                                 ctypes.c_void_p(s.cuda_stream)))


def dade_search_kernel_count(idx: Index, Q, K, nprobe, delta_d: int, ids, dists, *, max_K: int, max_nprobe: int,
                             workspace, offsets=None, **kw) -> int:
    """How many kernels dade_search with these arguments launches (captured
    into a CUDA graph, not run).  Keyword arguments as for dade_search; a
    workspace is required."""
    o = _opts(kw.pop("mode", "prune"), max_K, max_nprobe, kw.pop("first_wave", 0), kw.pop("tau", None),
              kw.pop("probe_in", None), kw.pop("probe_out", None), kw.pop("qrot_out", None), kw.pop("stats", None),
              kw.pop("status", None), workspace, kw.pop("wave_growth_log2", 0), kw.pop("final_test", False),
              kw.pop("estimator", "learned"), kw.pop("res_m", 8.0), kw.pop("test_steps", 0),
              kw.pop("scan_kernel", "auto"), kw.pop("candidate_budget_bytes", 0), kw.pop("queries_per_unit", 0))
    if kw:
        raise TypeError(f"unknown arguments {sorted(kw)}")
    n = ctypes.c_int64()
    _check(library().dade_search_kernel_count(idx.ptr, _ptr(Q), int(Q.shape[0]), _ptr(K), _ptr(nprobe),
                                              int(delta_d), ctypes.byref(o), _ptr(ids), _ptr(dists), _ptr(offsets),
                                              ctypes.byref(n)))
    return int(n.value)


def dade_search_noalloc(idx: Index, Q, K, nprobe, delta_d: int, ids, dists, *, max_K: int,
                        max_nprobe: int, mode: str = "prune", first_wave: int = 0, tau=None,
                        probe_in=None, probe_out=None, qrot_out=None, stats=None, status=None,
                        offsets=None, stream=None, wave_growth_log2: int = 0, final_test: bool = False,
                        estimator: str = "learned", res_m: float = 8.0, test_steps: int = 0,
                        scan_kernel: str = "auto", candidate_budget_bytes: int = 0,
                        queries_per_unit: int = 0) -> None:
    """dade_search whose scratch is the library's fixed device array: for
    callers that cannot allocate device memory.  Same arguments and results
    as dade_search except that no workspace is passed."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    o = _opts(mode, max_K, max_nprobe, first_wave, tau, probe_in, probe_out, qrot_out, stats, status, None,
              wave_growth_log2, final_test, estimator, res_m, test_steps, scan_kernel, candidate_budget_bytes,
              queries_per_unit)
    _check(library().dade_search_noalloc(idx.ptr, _ptr(Q), int(Q.shape[0]), _ptr(K), _ptr(nprobe),
                                         int(delta_d), ctypes.byref(o), _ptr(ids), _ptr(dists), _ptr(offsets),
                                         ctypes.c_void_p(s.cuda_stream)))


def dade_index_info_get(idx: Index) -> dict:
    info = L.IndexInfo()
    _check(library().dade_index_info_get(idx.ptr, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in L.IndexInfo._fields_}


def dade_index_centroids(idx: Index):
    info = dade_index_info_get(idx)
    out = np.empty((info["nlist"], info["D"]), np.float32)
    _check(library().dade_index_centroids(idx.ptr, out.ctypes.data))
    return out


def dade_index_assignment(idx: Index):
    info = dade_index_info_get(idx)
    out = np.empty(info["N"], np.int32)
    _check(library().dade_index_assignment(idx.ptr, out.ctypes.data))
    return out


def dade_index_list_sizes(idx: Index):
    info = dade_index_info_get(idx)
    out = np.empty(info["nlist"], np.int64)
    _check(library().dade_index_list_sizes(idx.ptr, out.ctypes.data))
    return out


def dade_index_stored(idx: Index, row0: int = 0, nrows: int | None = None):
    """Stored rotated vectors (slab precision, decoded to FP32) of input rows
    [row0, row0 + nrows): (nrows, D) host array."""
    info = dade_index_info_get(idx)
    nrows = info["N"] - int(row0) if nrows is None else int(nrows)
    out = np.empty((nrows, info["D"]), np.float32)
    _check(library().dade_index_stored(idx.ptr, int(row0), nrows, out.ctypes.data))
    return out


def dade_index_save(idx: Index, path: str) -> None:
    _check(library().dade_index_save(idx.ptr, str(path).encode()))


def dade_index_load(path: str) -> Index:
    out = ctypes.c_void_p()
    _check(library().dade_index_load(str(path).encode(), ctypes.byref(out)))
    return Index(out.value)


def dade_index_free(idx: Index) -> None:
    idx.close()


def dade_shard_owners(list_sizes, n_shards: int) -> np.ndarray:
    """Owner shard of each bucket (host computation; no device needed)."""
    sizes = np.ascontiguousarray(list_sizes, dtype=np.int64)
    out = np.empty(len(sizes), dtype=np.int32)
    _check(library().dade_shard_owners(sizes.ctypes.data, len(sizes), int(n_shards), out.ctypes.data))
    return out


def dade_index_shard(idx: Index, n_shards: int, shard: int) -> Index:
    """The index of one shard's buckets, on the current device."""
    out = ctypes.c_void_p()
    _check(library().dade_index_shard(idx.ptr, int(n_shards), int(shard), ctypes.byref(out)))
    return Index(out.value)


def dade_merge_topk(ids, dists, K, ids_out, dists_out, *, max_K: int, stream=None) -> None:
    """Merge per-part results: ids (int64) / dists (float32) CUDA tensors of
    n_parts x B x max_K, K a (B,) int32 CUDA tensor; outputs B x max_K."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    n_parts, B = int(ids.shape[0]), int(ids.shape[1])
    _check(library().dade_merge_topk(n_parts, B, int(max_K), _ptr(K), _ptr(ids), _ptr(dists), _ptr(ids_out),
                                     _ptr(dists_out), ctypes.c_void_p(s.cuda_stream)))


def dade_stage_timing(enable: bool, tensor_only: bool = False) -> None:
    """Event timing of the scan launches (all of them, or the tensor-core
    scan's alone) and their staged bytes."""
    _check(library().dade_stage_timing((2 if tensor_only else 1) if enable else 0))


def dade_stage_timing_read():
    """Returns (scan_ms, scan_launches, staged_bytes) since the last read."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    by = ctypes.c_double()
    _check(library().dade_stage_timing_read(ctypes.byref(ms), ctypes.byref(n), ctypes.byref(by)))
    return ms.value, n.value, by.value
