"""ctypes wrapper around the oracle refinement loop (``search.c``).

``prepare`` lays out an oracle index from FP64 inputs (rotation, centroids,
assignment); ``search`` runs the estimate / test / exact-distance loop of
Section V-B with one of the tau schedules; ``collect`` replays searches with
pruning off and records the per-step partial distances used to fit the
correction.  Test infrastructure only.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build
from . import ivf as _ivf
from . import pca as _pca
from . import storage as _storage

MODES = {"sequential": 0, "waves": 1, "frozen": 2}

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        _lib.oracle_search.restype = ctypes.c_int
        _lib.oracle_collect.restype = ctypes.c_int
        _lib.oracle_max_threads.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    _load().oracle_set_threads(ctypes.c_int(int(n)))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


# Relative slack of the test on the completed rotated distance: covers the
# FP32 rounding of the rotation and of the accumulated sums.
FINAL_REL = 1e-3


def n_steps(D: int, delta_d: int) -> int:
    """S = ceil(D / Delta_d): the number of Delta_d slabs covering D dims."""
    return -(-D // delta_d)


def disabled_tables(S: int):
    """Pruning off at every step: m1 = 0, beta = -inf."""
    return np.zeros(max(S - 1, 0)), np.full(max(S - 1, 0), -np.inf)


class OracleIndex:
    """Everything the oracle loop reads, in FP64 / original FP32."""

    def __init__(self, X, mu, R, centroids_r, assign, dtype="f32", ids=None, fp8_scale=None, flip_eps=None):
        self.X = np.ascontiguousarray(X, dtype=np.float32)
        self.N, self.D = self.X.shape
        self.mu = np.asarray(mu, dtype=np.float64)
        self.R = np.asarray(R, dtype=np.float64)
        self.C = np.asarray(centroids_r, dtype=np.float64)
        self.nlist = self.C.shape[0]
        self.assign = np.asarray(assign, dtype=np.int32)
        self.ids = (np.arange(self.N, dtype=np.int64) if ids is None
                    else np.ascontiguousarray(ids, dtype=np.int64))
        self.dtype = dtype
        Xr = _pca.rotate(self.X, self.mu, self.R)
        if dtype == "fp8" and fp8_scale is None:
            fp8_scale = _storage.fp8_scales(_storage.to_fp32(Xr))
        self.Xs = np.ascontiguousarray(_storage.stored(Xr, dtype, fp8_scale))
        # quantisation error norm ||x' - x~|| of each stored vector; FP32 and
        # FP64 storage count as exact (FINAL_REL covers their rounding)
        self.xerr = (np.zeros(self.N) if dtype in ("f32", "f64")
                     else np.ascontiguousarray(np.sqrt(((Xr - self.Xs) ** 2).sum(axis=1))))
        # sigma_i^2 of the RES bound: variance of each rotated dimension of the
        # indexed FP32 vectors (1/N)
        self.var = np.ascontiguousarray(_storage.to_fp32(Xr).astype(np.float64).var(axis=0))
        self.list_off, self.members = _ivf.lists_from_assignment(self.assign, self.nlist)
        # flip_eps: the rotation of another implementation may differ from
        # this one by up to e = flip_eps * ||x'|| per coordinate.  With BF16
        # or FP8 storage that can carry a value across a rounding midpoint of
        # the format (and, for FP8, move a per-dimension scale amax / 448 by
        # the largest e over the rows).  Xdev bounds, per coordinate, how far
        # the other side's stored value may then lie from Xs.
        self.Xdev = None
        if flip_eps is not None and dtype == "f32":
            # both sides round their own rotation to FP32: within e plus one
            # unit in the last place of the stored value
            rows = np.sqrt((Xr * Xr).sum(axis=1, keepdims=True))
            self.Xdev = np.ascontiguousarray(flip_eps * rows + np.spacing(np.abs(self.Xs).astype(np.float32))
                                             .astype(np.float64))
        if flip_eps is not None and dtype in ("bf16", "fp8"):
            self.Xdev = np.empty_like(self.Xs)
            rows = np.sqrt((Xr * Xr).sum(axis=1))
            if dtype == "fp8":
                s = np.asarray(fp8_scale, dtype=np.float64)
                amax = s * 448.0
                ds = np.where(amax > 0, flip_eps * rows.max() / np.where(amax > 0, amax, 1.0), 0.0)
            for a in range(0, self.N, 1 << 17):
                xr = Xr[a:a + (1 << 17)]
                xs = self.Xs[a:a + len(xr)]
                e = flip_eps * rows[a:a + len(xr), None]
                if dtype == "bf16":
                    lo = _storage.stored(xr - e, dtype)
                    hi = _storage.stored(xr + e, dtype)
                    dev = np.maximum(np.abs(lo - xs), np.abs(hi - xs))
                else:
                    dev = np.zeros_like(xs)
                    for sgn_x in (-1.0, 1.0):
                        for sgn_s in (-1.0, 1.0):
                            s2 = s * (1.0 + sgn_s * ds)
                            alt = _storage.stored(xr + sgn_x * e, dtype, s2.astype(np.float32))
                            dev = np.maximum(dev, np.abs(alt - xs))
                self.Xdev[a:a + len(xr)] = dev
        del Xr

    def rotate_queries(self, Q):
        return np.ascontiguousarray(_pca.rotate(Q, self.mu, self.R))

    def probe(self, Qr, nprobe: int):
        return _ivf.probe(Qr, self.C, nprobe)[0]


def search(idx: OracleIndex, Q, probes, nprobe, K, delta_d: int, m1, beta, mode="waves",
           first_wave: int = 1, tau=None, amb: float = 0.0, growth: int = 1, final_rel: float = np.inf,
           estimator: str = "learned", res_m: float = 8.0, ads_eps0: float = 2.1, pq=None, with_amb=False,
           uncertain_rows=None, qdev_eps=None, norm_eps: float = 0.0):
    """Returns (ids[B, Kmax], dists[B, Kmax], stats[B, 5]) where stats holds
    candidates visited, candidates pruned, exact distances taken, dims
    scanned, and candidates whose decision another rounding could flip:
    a test within amb * tau of its threshold (plus the effect of the
    index's Xdev, if any), for any tau the other side can hold once such
    decisions go the other way in earlier waves.  With with_amb, a fourth
    array amb_d[B] holds the smallest exact distance of such a candidate
    (+inf if none): below it, both sides' results hold the same entries.
    uncertain_rows (bool[N], rows in the index's order): rows the other side
    may represent otherwise (e.g. a product-quantisation code decided at a
    near tie); every decision on them counts as uncertain.  qdev_eps: the
    other side's rotated query may differ from this one's by up to
    qdev_eps * ||q'|| plus one FP32 unit per coordinate.  norm_eps: the
    other side computes dis' as ||q||^2 + ||x~||^2 - 2 <q, x~> (over the d
    dims so far), within norm_eps * max(d, 16) * (||q||^2 + ||x~||^2).  final_rel: the slack of the
    test on the completed rotated distance (FINAL_REL), or inf for no test.
    estimator "res": the Gaussian-bound test with multiplier res_m; "ads":
    the ADS test with parameter ads_eps0 (for both, m1 and beta are unused;
    None accepted); "pq": OPQ-L's single test m1 dis' + m3 e + beta > tau
    with pq = dict(codes[N, m] uint8, err[N], lut[B, m, 256], m1, m3, beta)
    (rows in the index's row order)."""
    lib = _load()
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    B = Q.shape[0]
    Qr = idx.rotate_queries(Q)
    Qdev = None
    if qdev_eps is not None:
        Qdev = np.ascontiguousarray(qdev_eps * np.sqrt((Qr * Qr).sum(axis=1, keepdims=True))
                                    + np.spacing(np.abs(Qr).astype(np.float32)).astype(np.float64))
    probes = np.ascontiguousarray(probes, dtype=np.int32)
    P = probes.shape[1]
    nprobe = np.ascontiguousarray(np.broadcast_to(np.asarray(nprobe, np.int32), (B,)))
    K = np.ascontiguousarray(np.broadcast_to(np.asarray(K, np.int32), (B,)))
    Kmax = int(K.max()) if B else 0
    S = n_steps(idx.D, delta_d)
    if m1 is None:
        m1, beta = np.zeros(max(S - 1, 0)), np.zeros(max(S - 1, 0))
    m1 = np.ascontiguousarray(m1, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    assert (m1.shape == (max(S - 1, 0),) or estimator == "pq") and beta.shape == m1.shape
    assert estimator in ("learned", "res", "ads", "pq")
    est = {"learned": 0, "res": 1, "ads": 2, "pq": 3}[estimator]
    est_param = res_m if estimator == "res" else ads_eps0
    pq_m, pq_codes, pq_err, pq_lut = 0, None, None, None
    if estimator == "pq":
        pq_codes = np.ascontiguousarray(pq["codes"], dtype=np.uint8)
        pq_m = pq_codes.shape[1]
        pq_err = np.ascontiguousarray(pq["err"], dtype=np.float64)
        pq_lut = np.ascontiguousarray(pq["lut"], dtype=np.float64)
        assert pq_codes.shape[0] == idx.N and pq_lut.shape == (B, pq_m, 256)
        m1 = np.array([pq["m1"]])
        beta = np.array([pq["beta"]])
        est_param = float(pq["m3"])
    tau_in = np.ascontiguousarray(np.full(B, np.inf) if tau is None else tau, dtype=np.float64)
    out_ids = np.empty((B, Kmax), dtype=np.int64)
    out_d = np.empty((B, Kmax))
    stats = np.zeros((B, 5), dtype=np.int64)
    amb_d = np.empty(B)
    unc_rows = None if uncertain_rows is None else np.ascontiguousarray(uncertain_rows, dtype=np.uint8)
    assert unc_rows is None or unc_rows.shape == (idx.N,)
    rc = lib.oracle_search(
        ctypes.c_int64(B), ctypes.c_int32(idx.D), ctypes.c_int32(delta_d), ctypes.c_int32(S),
        ctypes.c_int32(P), ctypes.c_int32(Kmax), ctypes.c_int32(MODES[mode]),
        ctypes.c_int32(first_wave), ctypes.c_int32(growth), ctypes.c_double(amb), ctypes.c_double(norm_eps),
        ctypes.c_double(final_rel),
        ctypes.c_int32(est), ctypes.c_double(est_param), _p(idx.var),
        ctypes.c_int32(pq_m), None if pq_codes is None else _p(pq_codes), None if pq_err is None else _p(pq_err),
        None if pq_lut is None else _p(pq_lut),
        _p(Qr), None if Qdev is None else _p(Qdev), _p(Q), _p(idx.Xs), None if idx.Xdev is None else _p(idx.Xdev),
        None if unc_rows is None else _p(unc_rows), _p(idx.xerr), _p(idx.X),
        _p(idx.ids),
        _p(idx.list_off), _p(idx.members), _p(probes), _p(nprobe), _p(K), _p(m1), _p(beta),
        _p(tau_in), _p(out_ids), _p(out_d), _p(stats), _p(amb_d))
    if rc != 0:
        raise ValueError("oracle_search rejected its arguments")
    if with_amb:
        return out_ids, out_d, stats, amb_d
    return out_ids, out_d, stats


def collect(idx: OracleIndex, Q, probes, nprobe, K, delta_d: int, first_wave: int = 1, growth: int = 1):
    """Replay with pruning off; returns a dict of per-candidate rows:
    partials[n, S-1], tau[n], dis[n], id[n], query[n]."""
    lib = _load()
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    B = Q.shape[0]
    Qr = idx.rotate_queries(Q)
    probes = np.ascontiguousarray(probes, dtype=np.int32)
    P = probes.shape[1]
    nprobe = np.ascontiguousarray(np.broadcast_to(np.asarray(nprobe, np.int32), (B,)))
    K = np.ascontiguousarray(np.broadcast_to(np.asarray(K, np.int32), (B,)))
    sizes = np.diff(idx.list_off)
    per_q = np.array([sizes[probes[b, :nprobe[b]]].sum() for b in range(B)], dtype=np.int64)
    row_off = np.zeros(B + 1, dtype=np.int64)
    np.cumsum(per_q, out=row_off[1:])
    n = int(row_off[-1])
    S = n_steps(idx.D, delta_d)
    partials = np.zeros((n, max(S - 1, 0)))
    tau = np.empty(n)
    dis = np.empty(n)
    ids = np.empty(n, dtype=np.int64)
    rc = lib.oracle_collect(
        ctypes.c_int64(B), ctypes.c_int32(idx.D), ctypes.c_int32(delta_d), ctypes.c_int32(S),
        ctypes.c_int32(P), ctypes.c_int32(first_wave), ctypes.c_int32(growth), _p(Qr), _p(Q), _p(idx.Xs),
        _p(idx.X),
        _p(idx.ids), _p(idx.list_off), _p(idx.members), _p(probes), _p(nprobe), _p(K),
        _p(row_off), _p(partials), _p(tau), _p(dis), _p(ids))
    if rc != 0:
        raise ValueError("oracle_collect rejected its arguments")
    query = np.repeat(np.arange(B, dtype=np.int64), per_q)
    return dict(partials=partials, tau=tau, dis=dis, id=ids, query=query, S=S)


def wave_bounds(nprobe: int, first_wave: int = 1, growth: int = 1):
    """Probe-rank boundaries of the WAVES schedule: 0, f, f 2^g, f 2^2g, ... capped."""
    b = [0]
    while b[-1] < nprobe:
        nxt = first_wave if b[-1] == 0 else b[-1] << min(growth, 40)
        b.append(min(nxt, nprobe))
    return b

