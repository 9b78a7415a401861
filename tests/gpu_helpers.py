"""Shared set-up of the GPU parity tests: oracle-made inputs (rotation,
centroids, assignment, correction tables) given to both the oracle and the
CUDA library, and a synchronous wrapper around the library's dade_search."""
import numpy as np

from oracle import fit, ivf, pca, search

# Half-width of the band (relative to tau) in which a learned test counts as
# ambiguous: a decision there may flip under the other side's rounding.
# "f32": the CUDA path rotates in FP32 (coordinate errors up to ~1e-5 on
# vectors of norm ~25 give partial-distance errors up to ~1.3e-5 tau);
# "bf16"/"fp8": stored values then differ by up to one unit of the format;
# "exact": both sides see bit-identical rotated inputs (pre-rotated data),
# leaving only FP32 accumulation, (8 + dims/8) ulps ~ 1.5e-6, plus tau's own.
AMB = {"f32": 3e-5, "bf16": 3e-5, "fp8": 3e-5, "exact": 5e-6}
# Per-coordinate bound, relative to ||x'||, of how far the device's rotation
# of a database vector may stray from the oracle's FP64 one (tcgen05 split-TF32
# GEMM with FP32 accumulation: measured <= 1.1e-6, see the stage-error test).
# With BF16 / FP8 slabs a coordinate that close to a rounding midpoint may be
# stored at the neighbouring value, and an FP8 scale (amax / 448) moves with
# the column maximum: the oracle's Xdev bounds both.
FLIP_EPS = 4e-6
# The tensor-core scan computes dis' = ||q||^2 + ||x~||^2 - 2 <q, x~> over the
# d dims so far (split TF32, FP32 accumulation); the oracle's slack for it is
# NORM_EPS * max(d, 16) * (||q||^2 + ||x~||^2): the dropped split terms
# (~2^-22 relative) and the accumulation rounding that grows with d.
NORM_EPS = 2e-8


def oracle_inputs(X, T, nlist, iters=8, seed=7, K=10, nprobe=8, delta_d=16, dtype="f32", r=0.995,
                  n_train=1000, prerotate=False):
    """Oracle PCA + k-means + fitted tables (rounded to FP32, as installed on
    the device).  Centroids are rounded to FP32 as well, so both sides probe
    with the same values.  With prerotate, the oracle's FP64 rotation is
    applied up front: both sides then get the FP32-rounded rotated vectors
    with R = I and mean = 0 (use rot() on queries)."""
    mu, R, lam = pca.train_rotation(X)
    if prerotate:
        X = pca.rotate(X, mu, R).astype(np.float32)
        T = pca.rotate(T, mu, R).astype(np.float32)
        rot = (lambda M, mu=mu, R=R: pca.rotate(M, mu, R).astype(np.float32))
        mu, R = np.zeros(X.shape[1]), np.eye(X.shape[1])
    else:
        rot = (lambda M: np.asarray(M, np.float32))
    Xr = pca.rotate(X, mu, R)
    init = np.random.default_rng(seed).choice(len(X), nlist, replace=False)
    C, a, _ = ivf.kmeans(Xr, init, iters)
    C32 = C.astype(np.float32)
    oidx = search.OracleIndex(X, mu, R, C32.astype(np.float64), a, dtype=dtype,
                              flip_eps=None if prerotate else FLIP_EPS)
    qdev = None if prerotate else FLIP_EPS
    m1, beta = fit_tables(oidx, T[:n_train], K, nprobe, delta_d, r)
    return dict(mu=mu, R=R, C32=C32, assign=a, oidx=oidx, m1=m1, beta=beta, X=X, rot=rot, qdev=qdev)


def fit_tables(oidx, T, K, nprobe, delta_d, r=0.995):
    pr = oidx.probe(oidx.rotate_queries(T), nprobe)
    S = search.n_steps(oidx.D, delta_d)
    rows = search.collect(oidx, T, pr, nprobe, K, delta_d)
    top, _, _ = search.search(oidx, T, pr, nprobe, K, delta_d, *search.disabled_tables(S))
    P, tau, lab = fit.label_rows(rows, top, cap=200_000)
    m1, beta, _ = fit.fit_correction(P, tau, lab, oidx.D, delta_d, r=r, min_label0=20)
    return m1.astype(np.float32), beta.astype(np.float32)


def build_gpu(G, X, inp, nlist, dtype="f32", delta_d=16):
    X = inp["X"] if X is None else X
    idx = G.ivf_build(X, inp["mu"], inp["R"], nlist, dtype=dtype, centroids=inp["C32"], assign=inp["assign"])
    G.dade_set_correction(idx, delta_d, inp["m1"], inp["beta"])
    return idx


def gpu_search(G, idx, Q, K, nprobe, delta_d, mode="prune", probe_in=None, tau=None, max_K=None,
               max_nprobe=None, first_wave=0, growth=0, final_test=False, estimator="learned", res_m=8.0,
               test_steps=0, want=(), scan_kernel="auto", candidate_budget_bytes=0, queries_per_unit=0):
    import torch
    B = Q.shape[0]
    Kv = np.broadcast_to(np.asarray(K, np.int32), (B,)).copy()
    Nv = np.broadcast_to(np.asarray(nprobe, np.int32), (B,)).copy()
    max_K = int(Kv.max()) if max_K is None else max_K
    max_nprobe = int(Nv.max()) if max_nprobe is None else max_nprobe
    dev = torch.device("cuda")
    q = torch.from_numpy(np.ascontiguousarray(Q, np.float32)).to(dev)
    k = torch.from_numpy(Kv).to(dev)
    n = torch.from_numpy(Nv).to(dev)
    ids = torch.full((B * max_K,), -7, dtype=torch.int64, device=dev)
    dists = torch.full((B * max_K,), -7.0, dtype=torch.float32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    extra = {}
    if "probes" in want:
        extra["probes"] = ("probe_out", torch.full((B, max_nprobe), -9, dtype=torch.int32, device=dev))
    if "qrot" in want:
        extra["qrot"] = ("qrot_out", torch.zeros((B, Q.shape[1]), dtype=torch.float32, device=dev))
    if "stats" in want:
        extra["stats"] = ("stats", torch.zeros((B, 4), dtype=torch.int64, device=dev))
    pin = None if probe_in is None else torch.from_numpy(np.ascontiguousarray(probe_in, np.int32)).to(dev)
    tin = None if tau is None else torch.from_numpy(np.ascontiguousarray(tau, np.float32)).to(dev)
    G.dade_search(idx, q, k, n, delta_d, ids, dists, max_K=max_K, max_nprobe=max_nprobe, mode=mode,
                  first_wave=first_wave, tau=tin, probe_in=pin, status=status, wave_growth_log2=growth,
                  final_test=final_test, estimator=estimator, res_m=res_m, test_steps=test_steps,
                  scan_kernel=scan_kernel, candidate_budget_bytes=candidate_budget_bytes,
                  queries_per_unit=queries_per_unit,
                  **{kw: t for kw, t in extra.values()})
    torch.cuda.synchronize()
    st = int(status.item())
    out = dict(ids=ids.view(B, max_K).cpu().numpy(), dists=dists.view(B, max_K).cpu().numpy(), status=st)
    for key, (_, v) in extra.items():
        out[key] = v.cpu().numpy()
    return out
