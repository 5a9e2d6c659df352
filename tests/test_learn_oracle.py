"""Pins of the hyperparameter-learning oracle (oracle/learn.py) to things
other than itself: closed forms of the mean extinction towards the
anticentre, the constant-density limit, the multivariate normal density of
scipy, derivatives in closed form, and recovery of the hyperparameters of
data drawn from the model itself.  CPU only."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O
from oracle import learn as Lr
from synth import make_disc_catalogue

THETA = np.array([2500.0, 150.0, 0.9e-3, 2200.0, 0.15])


def test_anticentre_mean_extinction_closed_form():
    """Towards l = 180 deg, b = 0: R = R_sun + t, z = 0, so the disc gives
    rho0 L (1 - exp(-s/L)); the bump integrates to A_b [Phi((s - s_b)/w) -
    Phi(-s_b/w)]."""
    s = np.array([50.0, 800.0, 2200.0, 4900.0])
    u = np.tile([-1.0, 0.0, 0.0], (len(s), 1))
    L, H, rho0, sb, Ab = THETA
    want = rho0 * L * (1 - np.exp(-s / L)) + Ab * (stats.norm.cdf((s - sb) / 400.0)
                                                   - stats.norm.cdf(-sb / 400.0))
    np.testing.assert_allclose(Lr.mean_extinction(u, s, THETA), want, rtol=1e-12)


def test_mean_extinction_is_line_integral_of_density():
    """Off the anticentre (disc and bump together), against a plain numerical
    line integral of the 3-D density."""
    l, b = np.radians([177.0, 184.5]), np.radians([0.03, -0.04])
    u = O.unit_vectors(l, b)
    s = np.array([1300.0, 4200.0])
    got = Lr.mean_extinction(u, s, THETA)
    for i in range(2):
        ref, _ = integrate.quad(lambda t: float(Lr.density(u[i] * t, THETA)), 0, s[i],
                                epsabs=0, epsrel=1e-12, limit=400, points=[2200.0])
        assert got[i] == pytest.approx(ref, rel=1e-10)


def test_constant_density_limit_gives_the_plain_prior_mean():
    """L, H -> infinity, A_b -> 0: m = ln(rho0 s) - K_ii/2, the prior mean of
    the constant-density model (gmead_oracle.build_cov)."""
    cat = make_disc_catalogue(60, truth="mean")
    cv = O.build_cov(cat, Q=16)
    u = O.unit_vectors(cat["l"], cat["b"])
    th = np.array([1e15, 1e15, cat["rho_bar"], 2000.0, 1e-30])
    m = Lr.prior_mean(u, cat["s"], th, cv["diag"])
    np.testing.assert_allclose(m, cv["m"], rtol=0, atol=1e-10)


def test_log_posterior_is_the_gaussian_marginal_likelihood_times_prior():
    rng = np.random.default_rng(0)
    n = 40
    A = rng.standard_normal((n, n))
    K = A @ A.T / n + 0.1 * np.eye(n)
    sig = rng.uniform(0.03, 0.1, n)
    m = rng.standard_normal(n)
    atil = m + rng.standard_normal(n)
    phi = np.log(THETA) + 0.1
    mu, s2 = Lr.prior_lognormal()
    want = stats.multivariate_normal(m, K + np.diag(sig ** 2)).logpdf(atil)
    want += stats.norm(mu, np.sqrt(s2)).logpdf(phi).sum()
    assert Lr.log_posterior(atil, sig, K, m, phi, mu, s2) == pytest.approx(want, rel=1e-12)


def test_hyperprior_has_the_stated_mean_and_sd():
    """Sect. 5: log-normal hyperpriors with standard deviation equal to mean."""
    mu, s2 = Lr.prior_lognormal()
    mean = np.exp(mu + s2 / 2)
    sd = np.sqrt((np.exp(s2) - 1) * np.exp(2 * mu + s2))
    np.testing.assert_allclose(mean, Lr.PRIOR_MEAN, rtol=1e-12)
    np.testing.assert_allclose(sd, Lr.PRIOR_MEAN, rtol=1e-12)


def test_jacobian_matches_closed_form_derivatives():
    """Anticentre, disc only in closed form: E = rho0 L (1 - e^{-s/L}) + bump;
    d ln E / d ln L, d ln E / d ln rho0, d/d ln A_b, d/d ln s_b by hand; H
    does not enter at z = 0."""
    s = np.array([300.0, 1500.0, 4000.0])
    u = np.tile([-1.0, 0.0, 0.0], (3, 1))
    L, H, rho0, sb, Ab = THETA
    w = 400.0
    e = np.exp(-s / L)
    disc = rho0 * L * (1 - e)
    Phi = stats.norm.cdf((s - sb) / w) - stats.norm.cdf(-sb / w)
    E = disc + Ab * Phi
    dL = L * (rho0 * (1 - e) - rho0 * (s / L) * e)
    dsb = sb * Ab * (-stats.norm.pdf((s - sb) / w) / w + stats.norm.pdf(-sb / w) / w)
    want = np.stack([dL / E, np.zeros(3), disc / E, dsb / E, Ab * Phi / E], axis=1)
    J = Lr.jacobian(u, s, THETA, np.zeros(3))
    np.testing.assert_allclose(J, want, rtol=1e-7, atol=1e-9)


def test_jacobian_is_the_derivative_of_the_prior_mean():
    """Off the anticentre, disc and bump together: against central
    differences of m in ln theta."""
    u = O.unit_vectors(np.radians([176.0, 183.0, 185.5]), np.radians([0.04, -0.02, 0.01]))
    s = np.array([600.0, 2100.0, 4600.0])
    J = Lr.jacobian(u, s, THETA, np.zeros(3))
    phi = np.log(THETA)
    for k in range(5):
        e = np.zeros(5)
        e[k] = 1e-5
        fd = (Lr.prior_mean(u, s, np.exp(phi + e), np.zeros(3))
              - Lr.prior_mean(u, s, np.exp(phi - e), np.zeros(3))) / 2e-5
        np.testing.assert_allclose(J[:, k], fd, rtol=1e-6, atol=1e-10)


def test_map_recovers_hyperparameters_of_model_draws():
    """Data drawn from the model itself, atil ~ N(m(theta), K + Sigma): over
    several draws the MAP lies within the Laplace errors of the truth (z
    scores of order one; a sign slip in the gradient or a wrong Hessian
    would bias or mis-scale them)."""
    cat = make_disc_catalogue(250, seed=3, truth="mean")
    cv = O.build_cov(cat, Q=16)
    K = cv["K"]
    u = O.unit_vectors(cat["l"], cat["b"])
    sig = cat["A_sigma"]
    m_true = Lr.prior_mean(u, cat["s"], THETA, np.diag(K))
    Lc = np.linalg.cholesky(K + np.diag(sig ** 2))
    z = []
    for seed in range(5):
        rng = np.random.default_rng(100 + seed)
        atil = m_true + Lc @ rng.standard_normal(len(sig))
        r = Lr.learn_mean(u, cat["s"], atil, sig, K, Lr.PRIOR_MEAN, max_iter=40, tol=1e-9)
        sd = np.sqrt(np.diag(r["cov_phi"]))
        zz = (r["phi"] - np.log(THETA)) / sd
        z.append(zz)
        # the mode: the Gauss-Newton gradient vanishes there
        assert r["iters"] < 40
    z = np.array(z)
    # well-constrained parameters: rho0, s_bump, A_bump (and L); H is prior-dominated
    assert np.all(np.abs(z) < 4.5), z
    assert 0.05 < np.mean(z[:, [0, 2, 3, 4]] ** 2) < 4.0, z
