"""Seeded mixtures standing in for the paper's datasets (Section VII-A).

The paper measures on public image/text embedding sets (SIFT, GIST, DEEP, ...)
that are not available here.  These generators draw data with the same
sizes, dimensionality, value range and power-law spectral decay instead:

* ``MixtureSpec``: a Gaussian mixture whose components share one covariance
  ``U^T diag(lam) U`` with ``lam_i ~ i^-alpha`` (normalised so that
  ``sum(lam) = D``) under a Haar-random orthogonal basis ``U``; component
  means are ``mean_scale * U^T (sqrt(lam) * z_k)`` with ``z_k ~ N(0, I)``;
  weights are uniform.  An optional affine map + clip + round produces
  SIFT-like integer vectors in [0, 255].
* ``VmfSpec``: L2-normalised vectors from a von Mises-Fisher-like mixture
  (random unit means, per-component concentration drawn uniformly), sampled
  with Wood's rejection method (Wood 1994, "Simulation of the von
  Mises-Fisher distribution").

Seeds (NumPy PCG64): data 1, queries 2, training queries 3, basis 4,
means 5.  Every array is float32 on return.
"""
from __future__ import annotations

import dataclasses

import numpy as np

SEED_DATA, SEED_QUERIES, SEED_TRAIN, SEED_BASIS, SEED_MEANS = 1, 2, 3, 4, 5


def power_law_spectrum(D: int, alpha: float) -> np.ndarray:
    """lam_i = c * i^-alpha for i = 1..D, scaled so that sum(lam) = D."""
    lam = np.arange(1, D + 1, dtype=np.float64) ** (-float(alpha))
    return lam * (D / lam.sum())


def haar_orthogonal(D: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian matrix with the
    signs of R's diagonal folded into Q (Mezzadri 2007)."""
    g = rng.standard_normal((D, D))
    q, r = np.linalg.qr(g)
    return q * np.sign(np.diag(r))[None, :]


@dataclasses.dataclass(frozen=True)
class MixtureSpec:
    D: int
    n_comp: int
    alpha: float
    mean_scale: float = 2.0
    # SIFT-like integer map: x -> clip(round(int_scale * x + int_offset), 0, 255)
    integer: bool = False
    int_scale: float = 48.0
    int_offset: float = 64.0

    def _basis(self):
        lam = power_law_spectrum(self.D, self.alpha)
        U = haar_orthogonal(self.D, np.random.default_rng(SEED_BASIS)).T  # rows = basis
        z = np.random.default_rng(SEED_MEANS).standard_normal((self.n_comp, self.D))
        means = self.mean_scale * (z * np.sqrt(lam)[None, :]) @ U
        return lam, U, means

    def population_covariance(self) -> np.ndarray:
        """Closed-form covariance of the (continuous, unmapped) mixture:
        shared covariance plus the covariance of the equally weighted means."""
        lam, U, means = self._basis()
        c = means - means.mean(axis=0, keepdims=True)
        return U.T @ np.diag(lam) @ U + c.T @ c / self.n_comp

    def sample(self, n: int, seed: int, chunk: int = 131072) -> np.ndarray:
        lam, U, means = self._basis()
        rng = np.random.default_rng(seed)
        out = np.empty((n, self.D), dtype=np.float32)
        sl = np.sqrt(lam)[None, :]
        for a in range(0, n, chunk):
            b = min(n, a + chunk)
            comp = rng.integers(0, self.n_comp, size=b - a)
            g = rng.standard_normal((b - a, self.D))
            x = means[comp] + (g * sl) @ U
            if self.integer:
                x = np.clip(np.rint(self.int_scale * x + self.int_offset), 0.0, 255.0)
            out[a:b] = x
        return out


@dataclasses.dataclass(frozen=True)
class VmfSpec:
    D: int
    n_comp: int
    kappa_lo: float = 20.0
    kappa_hi: float = 200.0

    def _params(self):
        rng = np.random.default_rng(SEED_MEANS)
        mu = rng.standard_normal((self.n_comp, self.D))
        mu /= np.linalg.norm(mu, axis=1, keepdims=True)
        kappa = rng.uniform(self.kappa_lo, self.kappa_hi, size=self.n_comp)
        return mu, kappa

    def sample(self, n: int, seed: int, chunk: int = 262144) -> np.ndarray:
        mu, kappa = self._params()
        rng = np.random.default_rng(seed)
        out = np.empty((n, self.D), dtype=np.float32)
        p = self.D
        for a in range(0, n, chunk):
            b = min(n, a + chunk)
            m = b - a
            comp = rng.integers(0, self.n_comp, size=m)
            k = kappa[comp]
            # Wood (1994): sample the cosine w to the mean direction by rejection.
            bb = (-2.0 * k + np.sqrt(4.0 * k * k + (p - 1.0) ** 2)) / (p - 1.0)
            x0 = (1.0 - bb) / (1.0 + bb)
            c = k * x0 + (p - 1.0) * np.log(1.0 - x0 * x0)
            w = np.empty(m)
            todo = np.arange(m)
            while todo.size:
                z = rng.beta((p - 1.0) / 2.0, (p - 1.0) / 2.0, size=todo.size)
                bt, xt, ct, kt = bb[todo], x0[todo], c[todo], k[todo]
                wt = (1.0 - (1.0 + bt) * z) / (1.0 - (1.0 - bt) * z)
                u = rng.uniform(size=todo.size)
                ok = kt * wt + (p - 1.0) * np.log(1.0 - xt * wt) - ct >= np.log(u)
                w[todo[ok]] = wt[ok]
                todo = todo[~ok]
            # direction orthogonal to the mean, uniform on the sub-sphere
            v = rng.standard_normal((m, p))
            mc = mu[comp]
            v -= (v * mc).sum(axis=1, keepdims=True) * mc
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            x = w[:, None] * mc + np.sqrt(np.maximum(0.0, 1.0 - w * w))[:, None] * v
            x /= np.linalg.norm(x, axis=1, keepdims=True)
            out[a:b] = x
        return out


# The workloads of the benchmark and tests.  Sizes follow the paper's
# datasets (Table "The Description of Datasets"): SIFT 1M x 128 integer
# descriptors, GIST 1M x 960, a 10M-vector normalised set, and a small case.
WORKLOADS = {
    "tiny": dict(spec=MixtureSpec(D=128, n_comp=16, alpha=1.0), N=10_000, n_queries=100,
                 n_train=2_000, nlist=64, nprobe=8, K=10, delta_d=16),
    # The mean spread 0.65 (in units of the shared per-dimension deviation)
    # makes IVF need nprobe ~32-64 of 4096 buckets for recall@10 ~0.95, as
    # IVF does on real SIFT1M; the default spread 2.0 separates the
    # components so well that nprobe 8 already reaches that recall.
    "sift1m": dict(spec=MixtureSpec(D=128, n_comp=256, alpha=0.8, integer=True, mean_scale=0.65),
                   N=1_000_000,
                   n_queries=10_000, n_train=10_000, nlist=4096, nprobe=64, K=100, delta_d=16),
    # The same spread for the GIST-shaped set: nprobe ~32-64 for recall@10
    # ~0.95 (measured at 1/10 scale with the same bucket size).
    "gist1m": dict(spec=MixtureSpec(D=960, n_comp=512, alpha=1.3, mean_scale=0.65), N=1_000_000, n_queries=1_000,
                   n_train=10_000, nlist=4096, nprobe=128, K=100, delta_d=32),
    "vmf10m": dict(spec=VmfSpec(D=96, n_comp=2048), N=10_000_000, n_queries=20_000,
                   n_train=10_000, nlist=4096, nprobe=256, K=100, delta_d=16),
    # The first index of the two-index serving mix (the second is gist1m).
    "serve2m": dict(spec=MixtureSpec(D=256, n_comp=256, alpha=1.0, mean_scale=0.65), N=2_000_000,
                    n_queries=20_000, n_train=10_000, nlist=4096, nprobe=64, K=100, delta_d=32),
}


def workload(name: str, N: int | None = None, n_queries: int | None = None,
             n_train: int | None = None):
    """Return (X, Q, T, cfg): database, queries and training queries for a
    named workload, optionally shrunk (N, n_queries, n_train)."""
    cfg = dict(WORKLOADS[name])
    spec = cfg["spec"]
    N = cfg["N"] if N is None else N
    nq = cfg["n_queries"] if n_queries is None else n_queries
    nt = cfg["n_train"] if n_train is None else n_train
    cfg.update(N=N, n_queries=nq, n_train=nt)
    X = spec.sample(N, SEED_DATA)
    Q = spec.sample(nq, SEED_QUERIES)
    T = spec.sample(nt, SEED_TRAIN)
    return X, Q, T, cfg
