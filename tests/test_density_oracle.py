"""Pins of the pseudo-density statement (oracle/density.py): the closed-form
truncated moments against Monte Carlo sampling of the paper's procedure
(sample the pair, keep samples whose farther extinction is larger) and
against their deterministic limit; the joint two-point predictive against the
textbook Gaussian conditional written with dense matrices, and against the
single-point predictive."""
import numpy as np
import pytest
from scipy import linalg

import oracle as O
from oracle import density as Dn
from synth import catalogue_subset, make_catalogue


@pytest.mark.parametrize("mu,S", [
    ([-1.0, -0.8], [[0.04, 0.03], [0.03, 0.05]]),
    ([-2.0, -2.05], [[0.10, 0.09], [0.09, 0.10]]),   # difference often negative
    ([0.3, 0.9], [[0.2, -0.05], [-0.05, 0.3]]),
])
def test_density_moments_against_sampling(mu, S, golden_kv):
    rng = np.random.default_rng(11)
    a = rng.multivariate_normal(mu, S, size=2_000_000)
    keep = a[:, 1] > a[:, 0]
    ds = golden_kv("sect5_setup.txt")["pair_offset_pc"][0]
    rho = (np.exp(a[keep, 1]) - np.exp(a[keep, 0])) / ds
    m, v = Dn.density_moments(mu, S, ds)
    se = rho.std() / np.sqrt(len(rho))
    assert abs(m - rho.mean()) < 5 * se
    assert v == pytest.approx(rho.var(), rel=0.02)


def test_density_moments_deterministic_limit():
    mu = np.array([-1.2, -1.1])
    S = 1e-12 * np.array([[1.0, 0.5], [0.5, 1.0]])
    m, v = Dn.density_moments(mu, S, 10.0)
    assert m == pytest.approx((np.exp(-1.1) - np.exp(-1.2)) / 10.0, rel=1e-6)
    assert abs(v) < 1e-12


@pytest.fixture(scope="module")
def field():
    cat = catalogue_subset(make_catalogue("c1_plain_400"), np.arange(160))
    cv = O.build_cov(cat)
    r = O.ep_run(cv["K"], cv["m"], cat["A_obs"], cat["A_sigma"], max_sweeps=3, tol=0.0)
    rng = np.random.default_rng(5)
    j = rng.choice(len(cat["s"]), 6, replace=False)
    lq, bq = cat["l"][j] + 1e-3, cat["b"][j] - 1e-3
    sq = cat["s"][j] * 0.9
    return cat, cv, r, lq, bq, sq


def test_pairs_marginals_equal_single_point_predictive(field):
    cat, cv, r, lq, bq, sq = field
    mu, cov = Dn.predict_pairs(cat, cv["K"], cv["m"], r["tau"], r["nu"], lq, bq, sq, 10.0)
    m1, v1 = O.predict(cat, cv["K"], cv["m"], r["tau"], r["nu"], lq, bq, sq)
    m2, v2 = O.predict(cat, cv["K"], cv["m"], r["tau"], r["nu"], lq, bq, sq + 10.0)
    np.testing.assert_allclose(mu[:, 0], m1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(mu[:, 1], m2, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(cov[:, 0, 0], v1, rtol=1e-10)
    np.testing.assert_allclose(cov[:, 1, 1], v2, rtol=1e-10)
    # two points 10 pc apart on one sightline stay positively correlated after
    # conditioning, and the 2 x 2 covariances are valid
    corr = cov[:, 0, 1] / np.sqrt(cov[:, 0, 0] * cov[:, 1, 1])
    assert np.all(corr > 0.0) and np.all(corr < 1.0)


def test_pairs_against_dense_gaussian_conditional(field, golden_kv):
    """Joint prior over (stars, near points, far points), the sites as noisy
    pseudo-observations nu/tau with variance 1/tau: the conditional of the
    query points by the textbook formula (no B = I + S^1/2 K S^1/2)."""
    cat, cv, r, lq, bq, sq = field
    ds = golden_kv("sect5_setup.txt")["pair_offset_pc"][0]
    mu, cov = Dn.predict_pairs(cat, cv["K"], cv["m"], r["tau"], r["nu"], lq, bq, sq, ds)
    assert np.all(r["tau"] > 0)
    nq = len(sq)
    # prior covariance blocks from the same sightline quadrature
    s = cat["s"]
    L0, sig2, c = float(cat["outer_scale_pc"]), float(cat["sigma2"]), float(cat["cutoff_pc"])
    Q = int(cat["n_nodes"])
    g = lambda rr: O.g_of_r(rr, sig2, L0)
    lp = np.concatenate([cat["l"], lq, lq])
    bp = np.concatenate([cat["b"], bq, bq])
    sp = np.concatenate([s, sq, sq + ds])
    up = O.unit_vectors(lp, bp)
    xp = up * sp[:, None]
    N = len(sp)
    C = np.zeros((N, N))
    for i in range(N):
        d = np.linalg.norm(xp - xp[i], axis=1)
        jj = np.flatnonzero(d <= c)
        chord2 = ((up[jj] - up[i]) ** 2).sum(1)
        v = O.K_from_R(O.pair_R(np.full(len(jj), sp[i]), sp[jj], chord2, g, Q), O.FORM_LOGNORMAL)
        C[i, jj] = v * np.where(jj == i, 1.0, O.wendland(d[jj] / c))
    C = 0.5 * (C + C.T)
    n = len(s)
    mprior = np.log(float(cat["rho_bar"]) * sp) - 0.5 * np.diag(C)
    Css, Cqs, Cqq = C[:n, :n], C[n:, :n], C[n:, n:]
    Nn = np.diag(1.0 / r["tau"])
    ytil = r["nu"] / r["tau"]
    G = linalg.solve(Css + Nn, np.column_stack([ytil - mprior[:n], Cqs.T]), assume_a="pos")
    mq = mprior[n:] + Cqs @ G[:, 0]
    Sq = Cqq - Cqs @ G[:, 1:]
    np.testing.assert_allclose(mu[:, 0], mq[:nq], rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(mu[:, 1], mq[nq:], rtol=1e-8, atol=1e-10)
    idx = np.arange(nq)
    np.testing.assert_allclose(cov[:, 0, 0], Sq[idx, idx], rtol=1e-7)
    np.testing.assert_allclose(cov[:, 1, 1], Sq[nq + idx, nq + idx], rtol=1e-7)
    np.testing.assert_allclose(cov[:, 0, 1], Sq[idx, nq + idx], rtol=1e-7)
