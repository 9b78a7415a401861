"""The C-ABI library loads and exports every entry point of include/dade.h,
and its host-only entry points (FP64 rotation, FP64 fit) agree with the
oracle.  No GPU is used."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dade.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("dade_", "ivf_"))))


@pytest.fixture(scope="module")
def lib():
    from paper_2404_16322_gb300 import build
    build.build()
    import paper_2404_16322_gb300 as G
    return G


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["dade_train_rotation", "ivf_build", "dade_fit_correction", "dade_search",
              "dade_index_save", "dade_index_load", "dade_index_free", "dade_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2404_16322_gb300 import _lib
    so = lib.library()
    for n in _declared():
        assert hasattr(so, n), n
        assert n in _lib.SIGNATURES, n
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    for n in _declared():
        assert n in exported, n  # C linkage, unmangled


def test_library_rotation_matches_oracle(lib, tiny):
    from oracle import pca
    mu, R, lam = lib.dade_train_rotation(tiny["X"])
    mu0, R0, lam0 = pca.train_rotation(tiny["X"])
    assert np.max(np.abs(R @ R.T - np.eye(len(R)))) < 1e-12
    assert np.allclose(mu, mu0, rtol=0, atol=1e-12 * np.abs(mu0).max())
    assert np.max(np.abs(lam - lam0)) < 1e-10 * lam0[0]
    gap = np.minimum(np.r_[lam0[:-1] - lam0[1:], np.inf], np.r_[np.inf, lam0[:-1] - lam0[1:]])
    ok = gap > 1e-6 * lam0[0]
    assert np.all(np.abs((R * R0).sum(1))[ok] > 1 - 1e-9)
    # same sign convention
    assert np.all((R * R0).sum(1)[ok] > 0)


def test_library_rotation_sampled_rows(lib):
    import synth
    X = synth.MixtureSpec(D=24, n_comp=4, alpha=1.0).sample(5000, 3)
    mu, R, lam = lib.dade_train_rotation(X, sample_n=1000, seed=9)
    assert np.max(np.abs(R @ R.T - np.eye(24))) < 1e-12
    assert np.all(np.diff(lam) <= 0)


def test_library_fit_matches_oracle_on_the_same_samples(lib, tiny):
    # Parity of the FP64 fit: both solvers on identical oracle-made samples.
    # The fitted values themselves have no closed form (parity unpinned for
    # the values); the two independent solvers must agree to 1e-6.
    from oracle import fit, search
    idx = search.OracleIndex(tiny["X"], tiny["mu"], tiny["R"], tiny["C"], tiny["assign"])
    T = tiny["T"][:500]
    pr = idx.probe(idx.rotate_queries(T), 8)
    rows = search.collect(idx, T, pr, 8, 10, 16)
    top, _, _ = search.search(idx, T, pr, 8, 10, 16, *search.disabled_tables(8))
    P, tau, lab = fit.label_rows(rows, top, cap=100_000)
    m1o, bo, info = fit.fit_correction(P, tau, lab, 128, 16, min_label0=20)
    m1l, bl = lib.dade_fit_samples(P, tau, lab, 128, 16, min_label0=20)
    en = np.isfinite(bo)
    assert np.array_equal(en, np.isfinite(bl))
    assert np.allclose(m1l, m1o, rtol=1e-6, atol=1e-9)
    assert np.allclose(bl[en], bo[en], rtol=1e-6, atol=1e-6 * np.abs(bo[en]).max())


def test_library_errors_are_status_codes(lib):
    from paper_2404_16322_gb300 import _lib
    with pytest.raises(_lib.DadeError) as e:
        lib.dade_train_rotation(np.zeros((1, 4), np.float32))
    assert e.value.status == 1 and "at least 2 rows" in str(e.value)
    with pytest.raises(_lib.DadeError):
        lib.dade_fit_samples(np.zeros((1, 7)), np.ones(1), np.zeros(1), 128, 12)


def test_library_random_rotation_is_orthogonal_seeded_and_haar(lib):
    R = lib.dade_random_rotation(40, seed=5)
    assert np.abs(R @ R.T - np.eye(40)).max() < 1e-12
    assert np.array_equal(R, lib.dade_random_rotation(40, seed=5))
    assert not np.allclose(R, lib.dade_random_rotation(40, seed=6))
    # Haar: every entry has mean 0 and variance 1/D; the determinant's sign
    # is +-1 with equal odds (a plain Householder Q without the sign fix has
    # a fixed pattern); the first row is uniform on the sphere, so its largest
    # |entry| has the distribution of a uniform direction's, compared here by
    # the mean against the oracle's numpy-made Haar rotations
    from oracle import pca
    D = 8
    Rs = np.stack([lib.dade_random_rotation(D, seed=s) for s in range(2000)])
    assert abs(Rs.mean()) < 4 / np.sqrt(Rs.size * D)
    assert abs(Rs.var() * D - 1) < 0.03
    dets = np.sign(np.linalg.det(Rs))
    assert 0.45 < np.mean(dets > 0) < 0.55
    ref = np.stack([pca.haar_rotation(D, s) for s in range(2000)])
    a, b = np.abs(Rs[:, 0]).max(1), np.abs(ref[:, 0]).max(1)
    assert abs(a.mean() - b.mean()) < 4 * np.sqrt(a.var() / len(a) + b.var() / len(b))
    # diagonal entries are not biased toward positive values
    assert abs(np.mean(Rs[:, np.arange(D), np.arange(D)])) < 4 / np.sqrt(2000 * D * D) * np.sqrt(D)


def test_library_ads_table_reproduces_the_oracle_ads_test(lib, tiny):
    # the installed table turns the learned test into ADS's: the oracle run
    # with the table as a learned test prunes exactly as the oracle's own ADS
    # test (decisions inside the FP32 rounding band of m1 excepted)
    from oracle import search
    idx = search.OracleIndex(tiny["X"], tiny["mu"], tiny["R"], tiny["C"], tiny["assign"])
    Q = tiny["Q"][:40]
    pr = idx.probe(idx.rotate_queries(Q), 8)
    for dd, e0 in [(16, 2.1), (32, 2.1), (8, 0.7)]:
        m1, beta = lib.dade_ads_table(128, dd, e0)
        assert m1.shape == (search.n_steps(128, dd) - 1,) and np.all(beta == 0)
        ads = search.search(idx, Q, pr, 8, 10, dd, None, None, estimator="ads", ads_eps0=e0, amb=1e-6)
        tab = search.search(idx, Q, pr, 8, 10, dd, m1.astype(np.float64), beta.astype(np.float64))
        un = ads[2][:, 4] == 0
        assert un.mean() > 0.9
        assert np.array_equal(ads[2][un, :4], tab[2][un, :4]), (dd, e0)
        assert ads[2][:, 1].sum() > 0
    with pytest.raises(Exception):
        lib.dade_ads_table(128, 16, -1.0)


def test_library_pq_fit_matches_oracle_on_the_same_samples(lib):
    # OPQ-L's three-feature classifier: the library's host FP64 fit and the
    # oracle's on identical samples (a boundary that needs the error feature)
    from oracle import fit
    rng = np.random.default_rng(8)
    n = 5000
    tau = rng.uniform(1.0, 2.0, n)
    dis = rng.uniform(0.0, 4.0, n)
    err = rng.uniform(0.0, 1.0, n)
    noise = rng.normal(0.0, 0.2, n)
    lab = (dis - 1.5 * err + noise > tau).astype(np.int8)
    m1o, m3o, bo, info = fit.fit_pq_correction(dis, err, tau, lab, r=0.995)
    m1l, m3l, bl = lib.dade_pq_fit_samples(dis, err, tau, lab, target_recall=0.995)
    assert info["enabled"]
    assert abs(m1l - m1o) <= 1e-6 * abs(m1o) and abs(m3l - m3o) <= 1e-6 * abs(m3o)
    assert abs(bl - bo) <= 1e-6 * max(1.0, abs(bo))
    # too few label-0 samples: disabled
    assert lib.dade_pq_fit_samples(dis[:50], err[:50], tau[:50], np.ones(50, np.int8))[2] == -np.inf


def test_library_random_rotation_sizes(lib):
    for D in (1, 2, 7, 960):
        R = lib.dade_random_rotation(D, seed=11)
        assert R.shape == (D, D)
        assert np.abs(R @ R.T - np.eye(D)).max() < 1e-11
    with pytest.raises(Exception):
        lib.dade_random_rotation(0)


def test_library_ads_table_edges(lib):
    # D not a multiple of delta_d: the last tested step covers min(s dd, D)
    m1, beta = lib.dade_ads_table(100, 32, 2.1)
    assert m1.shape == (3,) and np.all(beta == 0)
    d = np.array([32, 64, 96], dtype=np.float64)
    assert np.allclose(m1, (100 / d) / (1 + 2.1 / np.sqrt(d)), rtol=1e-6)
    # one step only: no test
    m1, beta = lib.dade_ads_table(16, 32, 2.1)
    assert m1.shape == (0,)
    # eps0 = 0: the plain scaled estimate against tau
    m1, _ = lib.dade_ads_table(64, 16, 0.0)
    assert np.allclose(m1, [4.0, 2.0, 4.0 / 3.0], rtol=1e-6)
