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
