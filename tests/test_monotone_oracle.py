"""Pins of the dA/ds >= 0 conditioning statement (oracle/monotone.py, exact
HMC for truncated Gaussians): the one-dimensional truncated normal's closed-
form moments, a two-point sightline against numerical integration, exact
feasibility of every sample, and the unconstrained limit."""
import numpy as np
import pytest
from scipy import integrate, stats

from oracle import monotone as M


def test_one_dimensional_truncated_normal_moments():
    rng = np.random.default_rng(1)
    mu, sd = 0.3, 1.2
    x = M.tmvn_hmc(np.array([mu]), np.array([[sd * sd]]), np.array([[1.0]]), np.array([0.0]),
                   np.array([1.0]), 40000, rng)
    a = -mu / sd
    lam = stats.norm.pdf(a) / (1 - stats.norm.cdf(a))
    mean = mu + sd * lam
    var = sd * sd * (1 + a * lam - lam * lam)
    assert np.all(x >= 0)
    assert x.mean() == pytest.approx(mean, abs=4 * np.sqrt(var / 40000) * 3)
    assert x.var() == pytest.approx(var, rel=0.05)


def test_two_point_sightline_against_integration():
    rng = np.random.default_rng(2)
    mu = np.array([-1.0, -1.05])            # the mean decreases: the constraint binds
    S = np.array([[0.04, 0.03], [0.03, 0.05]])
    x = M.monotone_sightline(mu, S, 40000, rng)
    assert np.all(x[:, 1] >= x[:, 0])
    pdf = stats.multivariate_normal(mu, S).pdf
    lo, hi = -3.0, 1.0
    Z = integrate.dblquad(lambda b, a: pdf([a, b]), lo, hi, lambda a: a, lambda a: hi)[0]
    m0 = integrate.dblquad(lambda b, a: a * pdf([a, b]), lo, hi, lambda a: a, lambda a: hi)[0] / Z
    m1 = integrate.dblquad(lambda b, a: b * pdf([a, b]), lo, hi, lambda a: a, lambda a: hi)[0] / Z
    assert x[:, 0].mean() == pytest.approx(m0, abs=0.01)
    assert x[:, 1].mean() == pytest.approx(m1, abs=0.01)


def test_unconstrained_limit_and_feasibility():
    rng = np.random.default_rng(3)
    m = 6
    mu = np.linspace(-2.0, 0.5, m)          # steeply increasing mean
    s = np.linspace(0, 1, m)
    S = 1e-3 * np.exp(-np.abs(s[:, None] - s[None, :]) / 0.5) + 1e-6 * np.eye(m)
    x = M.monotone_sightline(mu, S, 5000, rng)
    assert np.all(np.diff(x, axis=1) >= -1e-12)
    np.testing.assert_allclose(x.mean(axis=0), mu, atol=0.005)
    np.testing.assert_allclose(x.std(axis=0), np.sqrt(np.diag(S)), rtol=0.1)
