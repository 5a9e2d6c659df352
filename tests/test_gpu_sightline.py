"""Sightlines on the GPU against the oracle (oracle/monotone.py): the joint
predictive of the points of each sightline (gm_predict_sightlines) and the
dA/ds >= 0 sampler (gm_monotone_sample, exact HMC fed the oracle's momenta)."""
import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O
from oracle import monotone as M
from synth import catalogue_subset, make_catalogue

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_09705_gb300 import _build
    _build.build()
    import paper_1708_09705_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def field():
    cat = catalogue_subset(make_catalogue("c1_plain_400"), np.arange(200))
    cv = O.build_cov(cat)
    rng = np.random.default_rng(11)
    j = rng.choice(len(cat["s"]), 6, replace=False)
    lq, bq = cat["l"][j] + 2e-4, cat["b"][j] - 2e-4
    # 5 points per sightline; the widest spacing is beyond the cutoff
    sq = np.sort(cat["s"][j][:, None] * np.array([0.5, 0.7, 0.72, 0.9, 1.3])[None, :], axis=1)
    return cat, cv, lq, bq, sq


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sightline_predictive_matches_oracle(gm, field, prec):
    cat, cv, lq, bq, sq = field
    p = gm.PREC_FP64 if prec == "fp64" else gm.PREC_FP32
    cfg = gm.config_from_catalogue(cat, precision=p, cg_tol=1e-10 if prec == "fp64" else 1e-6)
    with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
        ctx.build_cov()
        ctx.ep_sweep(3, 0.0)
        tau, nu = ctx.get_sites()
        mean, cov = ctx.predict_sightlines(lq, bq, sq)
        # one point per sightline is the single-point predictive
        m1, c1 = ctx.predict_sightlines(lq, bq, sq[:, :1])
        mp, vp = ctx.predict(lq, bq, sq[:, 0])
        with pytest.raises(gm.GmError) as err:
            ctx.predict_sightlines(lq, bq, sq[:, ::-1])   # decreasing distances
        assert err.value.status == 1
    np.testing.assert_allclose(m1[:, 0], mp, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(c1[:, 0, 0], vp, rtol=1e-12)
    mu_o, S_o = M.sightline_predictive(cat, cv["K"], cv["m"], tau, nu, lq, bq, sq)
    assert np.array_equal(cov, np.transpose(cov, (0, 2, 1)))
    if prec == "fp64":
        np.testing.assert_allclose(mean, mu_o, rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(cov, S_o, rtol=1e-6, atol=1e-10)
    else:
        # the single-point predictive's FP32 bounds (1e-3 in ln A, 1e-2 in
        # variance); entries of points farther apart than the cutoff are only
        # the solve term (~1e-7 here), where the FP32 panel CG (relative
        # residual 1e-5) leaves absolute errors of a few 1e-7 (an FP32 CG
        # emulation on the CPU gave 4e-7): atol 5e-6
        np.testing.assert_allclose(mean, mu_o, atol=1e-3)
        np.testing.assert_allclose(cov, S_o, rtol=1e-2, atol=5e-6)


def _sampler_ctx(gm):
    cat = catalogue_subset(make_catalogue("c1_plain_400"), np.arange(50))
    cfg = gm.config_from_catalogue(cat)
    return gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"])


def test_sampler_matches_oracle_chain_on_predictives(gm, field):
    """The sampler fed the oracle's sightline predictives and momenta gives
    the oracle's chain (FP64 on both sides)."""
    cat, cv, lq, bq, sq = field
    r = O.ep_run(cv["K"], cv["m"], cat["A_obs"], cat["A_sigma"], max_sweeps=3, tol=0.0)
    mu, S = M.sightline_predictive(cat, cv["K"], cv["m"], r["tau"], r["nu"], lq, bq, sq)
    burn, ns = 10, 40
    mom = np.random.default_rng(5).standard_normal((len(lq), burn + ns, sq.shape[1]))
    with _sampler_ctx(gm) as ctx:
        out, hits = ctx.monotone_sample(mu, S, mom, burn)
    ref = np.array([M.monotone_sightline(mu[q], S[q], ns, None, burn=burn, momenta=mom[q])
                    for q in range(len(lq))])
    assert np.all(np.diff(out, axis=2) >= 0)
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-9)
    print("wall hits per sightline:", hits)


def _synthetic(rng, nsl, m):
    s = np.linspace(0.0, 1.0, m)
    base = np.exp(-np.abs(s[:, None] - s[None, :]) / 0.4)
    S = (0.02 + 0.03 * rng.random(nsl))[:, None, None] * base + 1e-4 * np.eye(m)
    mu = np.cumsum(rng.normal(0.0, 0.05, (nsl, m)), axis=1) - 1.0
    return mu, S


def test_sampler_many_sightlines(gm):
    """4096 sightlines of 16 points: every sample feasible and finite, and
    sampled sightlines equal to the oracle's chain."""
    rng = np.random.default_rng(6)
    nsl, m, burn, ns = 4096, 16, 10, 20
    mu, S = _synthetic(rng, nsl, m)
    mom = rng.standard_normal((nsl, burn + ns, m))
    with _sampler_ctx(gm) as ctx:
        out, hits = ctx.monotone_sample(mu, S, mom, burn)
    assert np.all(np.isfinite(out)) and np.all(np.diff(out, axis=2) >= 0)
    assert hits.min() > 0
    for q in rng.choice(nsl, 8, replace=False):
        ref = M.monotone_sightline(mu[q], S[q], ns, None, burn=burn, momenta=mom[q])
        np.testing.assert_allclose(out[q], ref, rtol=0, atol=1e-9)


def test_sampler_two_point_moments_against_integration(gm):
    """A binding constraint: the chain's means match the truncated bivariate
    normal's by numerical integration (independent of any sampler)."""
    mu = np.array([[-1.0, -1.05]])
    S = np.array([[[0.04, 0.03], [0.03, 0.05]]])
    n = 40000
    mom = np.random.default_rng(2).standard_normal((1, 50 + n, 2))
    with _sampler_ctx(gm) as ctx:
        x, _ = ctx.monotone_sample(mu, S, mom, 50)
    x = x[0]
    assert np.all(x[:, 1] >= x[:, 0])
    pdf = stats.multivariate_normal(mu[0], S[0]).pdf
    lo, hi = -3.0, 1.0
    Z = integrate.dblquad(lambda b, a: pdf([a, b]), lo, hi, lambda a: a, lambda a: hi)[0]
    m0 = integrate.dblquad(lambda b, a: a * pdf([a, b]), lo, hi, lambda a: a, lambda a: hi)[0] / Z
    m1 = integrate.dblquad(lambda b, a: b * pdf([a, b]), lo, hi, lambda a: a, lambda a: hi)[0] / Z
    assert x[:, 0].mean() == pytest.approx(m0, abs=0.01)
    assert x[:, 1].mean() == pytest.approx(m1, abs=0.01)


def test_sampler_edge_cases(gm):
    with _sampler_ctx(gm) as ctx:
        out, hits = ctx.monotone_sample(np.zeros((0, 3)), np.zeros((0, 3, 3)),
                                        np.zeros((0, 4, 3)), 1)
        assert out.shape == (0, 3, 3) and hits.shape == (0,)
        # burn-in only: hits counted, no samples
        mu, S = _synthetic(np.random.default_rng(1), 4, 5)
        out, hits = ctx.monotone_sample(mu, S, np.ones((4, 3, 5)), 3)
        assert out.shape == (4, 0, 5)
        # one point: no walls, each sample is mu + sd * momentum
        mom = np.random.default_rng(3).standard_normal((2, 5, 1))
        out, hits = ctx.monotone_sample(np.array([[0.3], [-1.2]]),
                                        np.array([[[0.25]], [[4.0]]]), mom, 1)
        assert np.all(hits == 0)
        np.testing.assert_allclose(out[:, :, 0],
                                   np.array([[0.3], [-1.2]]) + np.array([[0.5], [2.0]]) * mom[:, 1:, 0],
                                   atol=1e-15)
        # a covariance without a Cholesky factor, and a non-finite mean
        S_bad = S.copy()
        S_bad[2] = np.ones((5, 5))
        with pytest.raises(gm.GmError) as err:
            ctx.monotone_sample(mu, S_bad, np.ones((4, 3, 5)), 1)
        assert err.value.status == 4
        mu_bad = mu.copy()
        mu_bad[1, 2] = np.nan
        with pytest.raises(gm.GmError) as err:
            ctx.monotone_sample(mu_bad, S, np.ones((4, 3, 5)), 1)
        assert err.value.status == 6
