"""Oracle PCA rotation, FP64 (Section IV-B).

Theorem 1: among orthogonal projections, the principal-component matrix puts
the most variance in the leading (projected) dimensions and the least in the
residual ones, which by Eq. 2 minimises the variance of the estimation error
of a partial distance.  The Remark after it notes that the rotation makes the
covariance diagonal.  The data are centred first (footnote to Section IV-B).

Reading of the paper (it prints no recipe): mean over the sample; unbiased
covariance 1/(n-1) * sum (x-mu)(x-mu)^T; eigenvectors sorted by eigenvalue,
largest first; row i of R is the i-th eigenvector; each row's sign is fixed
so that its entry of largest magnitude (first such index on a tie) is
positive.  The eigendecomposition is LAPACK's symmetric solver via NumPy.
"""
from __future__ import annotations

import numpy as np


def train_rotation(X: np.ndarray):
    """Return (mean[D], R[D, D], eigvals[D]) in FP64 for the rows of X."""
    Xd = np.asarray(X, dtype=np.float64)
    n = Xd.shape[0]
    mu = Xd.mean(axis=0)
    Xc = Xd - mu
    C = Xc.T @ Xc / (n - 1)
    lam, V = np.linalg.eigh(C)  # ascending
    order = np.argsort(-lam, kind="stable")
    lam = lam[order]
    R = V[:, order].T.copy()
    piv = np.argmax(np.abs(R), axis=1)
    sgn = np.sign(R[np.arange(R.shape[0]), piv])
    sgn[sgn == 0] = 1.0
    R *= sgn[:, None]
    return mu, R, lam


def rotate(X: np.ndarray, mu: np.ndarray, R: np.ndarray) -> np.ndarray:
    """x' = R (x - mu), FP64 (Section IV-A: x_D = R x, after centring)."""
    return (np.asarray(X, dtype=np.float64) - mu) @ np.asarray(R, dtype=np.float64).T


def haar_rotation(D: int, seed: int) -> np.ndarray:
    """A random orthogonal R[D, D] from the Haar measure, FP64: the random
    rotation of ADS (Section III, Distance Estimation).  Q from the QR
    decomposition of a standard Gaussian matrix, with each column's sign set
    by the sign of R's diagonal entry so that the distribution is exactly
    Haar (Mezzadri, "How to generate random matrices from the classical
    compact groups", 2007).  Returned as rows (x' = R x)."""
    G = np.random.default_rng(seed).standard_normal((D, D))
    Qm, Rm = np.linalg.qr(G)
    s = np.sign(np.diag(Rm))
    s[s == 0] = 1.0
    return (Qm * s[None, :]).T.copy()
