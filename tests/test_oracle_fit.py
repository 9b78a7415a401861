"""Pins of the oracle's data-driven correction (Section V-A, V-B, VII-A)."""
import math

import numpy as np
import pytest
from scipy import optimize

from oracle import fit, search


def test_splitmix64_published_first_output():
    # SplitMix64 from state 0: first output 0xE220A8397B1DCDAF
    # (Steele, Lea, Flood 2014 reference generator).
    assert int(fit.splitmix64(np.array([0], dtype=np.uint64))[0]) == 0xE220A8397B1DCDAF


def test_sample_uniform_range_and_mean():
    u = fit.sample_uniform(3, np.arange(200_000) % 97, np.arange(200_000))
    assert u.min() >= 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.005


def _two_class(n=4000, seed=0, sep=1.0):
    rng = np.random.default_rng(seed)
    y = (rng.random(n) < 0.4).astype(np.float64)
    F = rng.standard_normal((n, 2)) + sep * np.column_stack([y, -y])
    return F, y


def test_irls_matches_an_independent_quasi_newton_solver():
    F, y = _two_class()
    theta, it, g = fit.fit_logistic(F, y)
    assert g < 1e-10

    def f(t):
        z = F @ t[:2] + t[2]
        return np.mean(np.logaddexp(0, z) - y * z) + 0.5e-8 * (t[0] ** 2 + t[1] ** 2)

    ref = optimize.minimize(f, np.zeros(3), method="BFGS", options=dict(gtol=1e-12))
    assert np.allclose(theta, ref.x, rtol=1e-5, atol=1e-6)


def test_irls_separable_boundary_between_classes():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((100, 2)) * 0.3 + [3, 0]
    b = rng.standard_normal((100, 2)) * 0.3 + [-3, 0]
    F = np.concatenate([a, b])
    y = np.r_[np.ones(100), np.zeros(100)]
    theta, _, _ = fit.fit_logistic(F, y)
    z = F @ theta[:2] + theta[2]
    assert np.all(z[:100] > 0) and np.all(z[100:] < 0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_beta_prime_closed_form_equals_bisection(seed):
    rng = np.random.default_rng(seed)
    v = np.round(rng.standard_normal(3001) * 50, 1)  # with ties
    for r in [0.9, 0.99, 0.995, 0.9999]:
        a = fit.beta_prime_closed_form(v, r)
        b = fit.beta_prime_bisection(v, r)
        assert a == b or np.nextafter(b, np.inf) == a or np.nextafter(a, np.inf) == b
        assert 1 - np.count_nonzero(v < a) / len(v) >= r


def test_beta_prime_known_answer():
    v = np.arange(1, 1001, dtype=np.float64)
    # f = floor(0.01 * 1000) = 10 allowed prunes -> beta' = v_(11) = 11
    assert fit.beta_prime_closed_form(v, 0.99) == 11.0


def test_fit_correction_on_tiny_meets_per_step_recall_and_nests(tiny):
    idx = search.OracleIndex(tiny["X"], tiny["mu"], tiny["R"], tiny["C"], tiny["assign"])
    T = tiny["T"][:600]
    pr = idx.probe(idx.rotate_queries(T), 8)
    S = search.n_steps(128, 16)
    rows = search.collect(idx, T, pr, 8, 10, 16)
    top, _, _ = search.search(idx, T, pr, 8, 10, 16, *search.disabled_tables(S))
    P, tau, lab = fit.label_rows(rows, top, cap=50_000)
    # label semantics: label 1 means dis > tau
    assert np.all(np.isfinite(tau))
    m1, beta, info = fit.fit_correction(P, tau, lab, 128, 16, r=0.995, min_label0=20)
    r_s = 1 - 0.005 / S
    active = np.ones(len(tau), bool)
    for s in range(1, S):
        pruned = m1[s - 1] * P[:, s - 1] + beta[s - 1] > tau
        l0 = active & (lab == 0)
        if l0.sum():
            assert 1 - (pruned & l0).sum() / l0.sum() >= r_s - 1e-12
        new = active & ~pruned
        assert np.all(new <= active)
        active = new
    assert any(r["enabled"] for r in info)
    for r in info:
        if r["enabled"]:
            assert r["grad"] < 1e-10 and r["w2"] < 0


def test_label_rows_semantics():
    rows = dict(partials=np.zeros((5, 1)), tau=np.array([np.inf, 5, 5, 5, 5.0]),
                dis=np.array([1, 2, 6, 4, 5.0]), id=np.arange(5), query=np.zeros(5, np.int64))
    top = np.array([[0, 1]])
    P, tau, lab = fit.label_rows(rows, top)
    # row 0: tau inf -> dropped; row 1: in top -> label 0; row 2: 6 > 5 ->
    # label 1; rows 3, 4: dis <= tau but not in top -> dropped.
    assert list(lab) == [0, 1] and list(tau) == [5, 5]
    assert math.isfinite(tau.sum())
