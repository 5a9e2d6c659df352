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


# ------------------------------------------------- sightline joint predictive
import oracle as O  # noqa: E402
from scipy import linalg  # noqa: E402
from oracle import density as Dn  # noqa: E402
from synth import catalogue_subset, make_catalogue  # noqa: E402


@pytest.fixture(scope="module")
def field():
    cat = catalogue_subset(make_catalogue("c1_plain_400"), np.arange(160))
    cv = O.build_cov(cat)
    r = O.ep_run(cv["K"], cv["m"], cat["A_obs"], cat["A_sigma"], max_sweeps=3, tol=0.0)
    rng = np.random.default_rng(8)
    j = rng.choice(len(cat["s"]), 4, replace=False)
    lq, bq = cat["l"][j] + 1e-3, cat["b"][j] - 1e-3
    # 5 points per sightline, spacings from well inside to beyond the cutoff
    sq = np.sort(cat["s"][j][:, None] * np.array([0.5, 0.7, 0.72, 0.9, 1.3])[None, :], axis=1)
    return cat, cv, r, lq, bq, sq


def test_sightline_marginals_equal_single_point_predictive(field):
    cat, cv, r, lq, bq, sq = field
    mu, cov = M.sightline_predictive(cat, cv["K"], cv["m"], r["tau"], r["nu"], lq, bq, sq)
    m1, v1 = O.predict(cat, cv["K"], cv["m"], r["tau"], r["nu"], np.repeat(lq, 5),
                       np.repeat(bq, 5), sq.reshape(-1))
    np.testing.assert_allclose(mu.reshape(-1), m1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(np.diagonal(cov, axis1=1, axis2=2).reshape(-1), v1, rtol=1e-10)
    for q in range(len(lq)):
        np.testing.assert_array_equal(cov[q], cov[q].T)
        assert np.linalg.eigvalsh(cov[q]).min() > 0


def test_sightline_two_points_equal_pair_predictive(field):
    cat, cv, r, lq, bq, sq = field
    s2 = np.stack([sq[:, 0], sq[:, 0] + 10.0], axis=1)
    mu, cov = M.sightline_predictive(cat, cv["K"], cv["m"], r["tau"], r["nu"], lq, bq, s2)
    mp, cp = Dn.predict_pairs(cat, cv["K"], cv["m"], r["tau"], r["nu"], lq, bq, sq[:, 0], 10.0)
    np.testing.assert_allclose(mu, mp, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(cov, cp, rtol=1e-10, atol=1e-14)


def test_sightline_without_sites_is_the_prior_block_of_K(field):
    """Zero sites: the predictive is the prior, whose mean and covariance must
    equal the covariance assembly of a catalogue made of the points."""
    cat, cv, r, lq, bq, sq = field
    n = len(cat["s"])
    mu, cov = M.sightline_predictive(cat, cv["K"], cv["m"], np.zeros(n), np.zeros(n), lq, bq, sq)
    for q in range(len(lq)):
        pts = dict(cat, l=np.full(5, lq[q]), b=np.full(5, bq[q]), s=sq[q])
        pc = O.build_cov(pts)
        np.testing.assert_allclose(mu[q], pc["m"], rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(cov[q], pc["K"], rtol=1e-12, atol=1e-15)
    # the widest spacing (factor 1.3 / 0.5 of the distance) is beyond the cutoff
    assert np.any(cov[:, 0, 4] == 0.0)


def test_sightline_against_dense_gaussian_conditional(field):
    """Joint prior over (stars, all sightline points) from one covariance
    assembly, sites as noisy pseudo-observations nu/tau with variance 1/tau:
    the textbook conditional (no B = I + S^1/2 K S^1/2)."""
    cat, cv, r, lq, bq, sq = field
    mu, cov = M.sightline_predictive(cat, cv["K"], cv["m"], r["tau"], r["nu"], lq, bq, sq)
    n, nsl, Mp = len(cat["s"]), len(lq), sq.shape[1]
    allc = dict(cat, l=np.concatenate([cat["l"], np.repeat(lq, Mp)]),
                b=np.concatenate([cat["b"], np.repeat(bq, Mp)]),
                s=np.concatenate([cat["s"], sq.reshape(-1)]))
    ac = O.build_cov(allc)
    C, mprior = ac["K"], ac["m"]
    Css, Cqs, Cqq = C[:n, :n], C[n:, :n], C[n:, n:]
    G = linalg.solve(Css + np.diag(1.0 / r["tau"]),
                     np.column_stack([r["nu"] / r["tau"] - mprior[:n], Cqs.T]), assume_a="pos")
    mq = mprior[n:] + Cqs @ G[:, 0]
    Sq = Cqq - Cqs @ G[:, 1:]
    np.testing.assert_allclose(mu.reshape(-1), mq, rtol=1e-8, atol=1e-10)
    for q in range(nsl):
        blk = slice(q * Mp, (q + 1) * Mp)
        np.testing.assert_allclose(cov[q], Sq[blk, blk], rtol=1e-7, atol=1e-12)


def test_given_momenta_reproduce_the_rng_chain():
    """Passing the draws explicitly gives the same chain as drawing them."""
    mu = np.array([-1.0, -1.05, -0.9])
    S = np.array([[0.04, 0.03, 0.02], [0.03, 0.05, 0.03], [0.02, 0.03, 0.06]])
    a = M.monotone_sightline(mu, S, 30, np.random.default_rng(4), burn=5)
    mom = np.random.default_rng(4).standard_normal((35, 3))
    b = M.monotone_sightline(mu, S, 30, None, burn=5, momenta=mom)
    np.testing.assert_array_equal(a, b)
