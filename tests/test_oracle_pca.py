"""Pins of the oracle's PCA rotation (Section IV-B, Theorem 1, the Remark on
decorrelation) against properties the mathematics fixes."""
import numpy as np

import synth
from oracle import pca


def _data(n=20_000, D=48, comps=6, alpha=1.0):
    spec = synth.MixtureSpec(D=D, n_comp=comps, alpha=alpha)
    return spec, spec.sample(n, 11)


def test_rotation_is_orthogonal():
    _, X = _data()
    _, R, _ = pca.train_rotation(X)
    assert np.max(np.abs(R @ R.T - np.eye(R.shape[0]))) < 1e-12


def test_eigenvalues_descending_and_sum_to_trace():
    _, X = _data()
    _, _, lam = pca.train_rotation(X)
    assert np.all(np.diff(lam) <= 0)
    assert lam[-1] >= -1e-12 * lam[0]
    # trace of the covariance = sum of per-column sample variances
    tr = np.var(X.astype(np.float64), axis=0, ddof=1).sum()
    assert abs(lam.sum() - tr) <= 1e-10 * tr


def test_rotated_coordinates_are_decorrelated_with_variances_lambda():
    # The Remark after Theorem 1: the rotation removes the off-diagonal
    # covariance; the variance of rotated coordinate i is lambda_i.  A
    # transposed R (columns instead of rows) fails this.
    _, X = _data()
    mu, R, lam = pca.train_rotation(X)
    Xr = pca.rotate(X, mu, R)
    C = np.cov(Xr, rowvar=False)
    off = C - np.diag(np.diag(C))
    assert np.max(np.abs(off)) < 1e-10 * lam[0]
    assert np.allclose(np.diag(C), lam, rtol=1e-9, atol=1e-12 * lam[0])
    assert np.max(np.abs(Xr.mean(axis=0))) < 1e-9 * np.sqrt(lam[0])


def test_full_dimension_rotated_distance_equals_original():
    _, X = _data(n=2000)
    mu, R, _ = pca.train_rotation(X)
    Xr = pca.rotate(X, mu, R)
    a, b = X[:500].astype(np.float64), X[500:1000].astype(np.float64)
    d0 = ((a - b) ** 2).sum(1)
    d1 = ((Xr[:500] - Xr[500:1000]) ** 2).sum(1)
    assert np.max(np.abs(d1 - d0) / d0) < 1e-9


def test_sign_rule_largest_entry_positive():
    _, X = _data(n=3000)
    _, R, _ = pca.train_rotation(X)
    piv = np.argmax(np.abs(R), axis=1)
    assert np.all(R[np.arange(len(R)), piv] > 0)


def test_sample_spectrum_matches_population_closed_form():
    # The generator's covariance is known in closed form (shared covariance
    # plus the covariance of the component means).  Sample eigenvalues must
    # agree with its eigenvalues within the O(lambda_1 sqrt(D / n)) bound of
    # eigenvalue perturbation (Weyl), and the leading eigenvector with the
    # population's when its eigengap is large.
    spec, X = _data(n=100_000, D=32, comps=8, alpha=1.2)
    _, R, lam = pca.train_rotation(X)
    Cp = spec.population_covariance()
    lp, Vp = np.linalg.eigh(Cp)
    lp, Vp = lp[::-1], Vp[:, ::-1]
    bound = 3.0 * lp[0] * np.sqrt(32 / 100_000)
    assert np.max(np.abs(lam - lp)) < bound
    gap = lp[0] - lp[1]
    if gap > 0.2 * lp[0]:
        assert abs(R[0] @ Vp[:, 0]) > 0.99
