"""Pins of the block-site PIC-EP statement (oracle/pic.py, the simplified case
of Sect. 4.1): reductions to exact GP regression (inducing points at every
star; a single block), to independent blocks (inducing point out of reach),
and EP against one direct linear-Gaussian conditioning of the PITC model."""
import numpy as np
import pytest

import oracle as O
from oracle import pic as P
from synth import catalogue_subset, make_catalogue


@pytest.fixture(scope="module")
def setup():
    cat = make_catalogue("c1_plain_400", truth="mean")
    cat = catalogue_subset(cat, np.arange(120))
    n = len(cat["s"])
    rng = np.random.default_rng(8)
    # inducing points: 20 positions inside the field, plus one far away
    li = rng.uniform(cat["l"].min(), cat["l"].max(), 20)
    bi = rng.uniform(cat["b"].min(), cat["b"].max(), 20)
    si = np.exp(rng.uniform(np.log(150), np.log(2500), 20))
    union = dict(cat)
    for k, extra in (("l", li), ("b", bi), ("s", si)):
        union[k] = np.concatenate([cat[k], extra, [cat[k].mean()] if k != "s" else [20000.0]])
    union["A_obs"] = np.zeros(len(union["s"]))
    union["A_sigma"] = np.ones(len(union["s"]))
    cv = O.build_cov(union)
    K, m = cv["K"], cv["m"]
    A = np.clip(cat["A_obs"], 0.02, None)
    atil = np.log(A) + 0.02 * rng.standard_normal(n)
    sig2 = (cat["A_sigma"] / A) ** 2
    order = np.argsort(cat["l"])
    blocks_idx = np.array_split(order, 4)
    return dict(n=n, K=K, m=m, atil=atil, sig2=sig2, blocks_idx=blocks_idx,
                ind=np.arange(n, n + 20), far=np.array([n + 20]))


def make_blocks(S, u_idx, groups):
    K, m = S["K"], S["m"]
    return [dict(Kku=K[np.ix_(g, u_idx)], Kkk=K[np.ix_(g, g)], m=m[g], atil=S["atil"][g],
                 sig2=S["sig2"][g], idx=g) for g in groups]


def predict_stars(S, u_idx, blocks, post_mean, post_cov):
    K, m = S["K"], S["m"]
    mu = np.empty(S["n"])
    var = np.empty(S["n"])
    for b in blocks:
        g = b["idx"]
        mm, vv = P.pic_predict(K[np.ix_(u_idx, u_idx)], m[u_idx], post_mean, post_cov, b,
                               K[np.ix_(g, u_idx)], np.diag(K)[g], K[np.ix_(g, g)], m[g])
        mu[g], var[g] = mm, vv
    return mu, var


def exact(S, idx):
    K = S["K"][np.ix_(idx, idx)]
    return O.gp_regression(K, S["m"][idx], S["atil"][idx], S["sig2"][idx])


def test_inducing_points_at_every_star_give_exact_gp(setup):
    S = setup
    u_idx = np.arange(S["n"])
    blocks = make_blocks(S, u_idx, S["blocks_idx"])
    Kuu = S["K"][np.ix_(u_idx, u_idx)]
    pm, pc, _ = P.ep_blocks(Kuu, blocks, S["m"][u_idx], max_sweeps=2)
    mean, var = exact(S, u_idx)
    np.testing.assert_allclose(pm, mean, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(np.diag(pc), var, rtol=1e-7)
    mu, v = predict_stars(S, u_idx, blocks, pm, pc)
    np.testing.assert_allclose(mu, mean, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(v, var, rtol=1e-6, atol=1e-12)


def test_single_block_is_exact_for_any_inducing_set(setup):
    S = setup
    u_idx = S["ind"]
    allg = [np.arange(S["n"])]
    blocks = make_blocks(S, u_idx, allg)
    Kuu = S["K"][np.ix_(u_idx, u_idx)]
    pm, pc, _ = P.ep_blocks(Kuu, blocks, S["m"][u_idx], max_sweeps=2)
    mu, v = predict_stars(S, u_idx, blocks, pm, pc)
    mean, var = exact(S, np.arange(S["n"]))
    np.testing.assert_allclose(mu, mean, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(v, var, rtol=1e-6)


def test_unreachable_inducing_point_gives_independent_blocks(setup):
    """The paper's block-diagonal limit (an empty inducing set): an inducing
    point beyond the cutoff of every star couples nothing."""
    S = setup
    u_idx = S["far"]
    assert np.all(S["K"][np.ix_(np.arange(S["n"]), u_idx)] == 0.0)
    blocks = make_blocks(S, u_idx, S["blocks_idx"])
    Kuu = S["K"][np.ix_(u_idx, u_idx)]
    pm, pc, _ = P.ep_blocks(Kuu, blocks, S["m"][u_idx], max_sweeps=2)
    mu, v = predict_stars(S, u_idx, blocks, pm, pc)
    for g in S["blocks_idx"]:
        mean, var = exact(S, g)
        np.testing.assert_allclose(mu[g], mean, rtol=1e-8, atol=1e-10)
        np.testing.assert_allclose(v[g], var, rtol=1e-6)


def test_ep_reaches_the_pitc_posterior_in_one_sweep(setup):
    S = setup
    u_idx = S["ind"]
    blocks = make_blocks(S, u_idx, S["blocks_idx"])
    Kuu = S["K"][np.ix_(u_idx, u_idx)]
    pm, pc, hist = P.ep_blocks(Kuu, blocks, S["m"][u_idx], max_sweeps=3)
    dm, dc = P.pitc_posterior_direct(Kuu, blocks, S["m"][u_idx])
    np.testing.assert_allclose(pm, dm, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(pc, dc, rtol=1e-7, atol=1e-12)
    for (L1, e1), (L2, e2) in zip(hist[0], hist[1]):
        np.testing.assert_allclose(L2, L1, rtol=1e-8, atol=1e-9 * np.abs(L1).max())
        np.testing.assert_allclose(e2, e1, rtol=1e-8, atol=1e-9 * np.abs(e1).max())
