"""PITC / PIC posterior over inducing points on the GPU (gm_pic_posterior)
against oracle/pic.py."""
import numpy as np
import pytest

import oracle as O
from oracle import pic as P
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


def test_pic_posterior_matches_oracle(gm):
    cat = catalogue_subset(make_catalogue("c1_plain_400", truth="mean"), np.arange(300))
    n = len(cat["s"])
    rng = np.random.default_rng(9)
    R = 40
    li = rng.uniform(cat["l"].min(), cat["l"].max(), R)
    bi = rng.uniform(cat["b"].min(), cat["b"].max(), R)
    si = np.exp(rng.uniform(np.log(150), np.log(2500), R))
    union = dict(cat, l=np.concatenate([cat["l"], li]), b=np.concatenate([cat["b"], bi]),
                 s=np.concatenate([cat["s"], si]))
    cv = O.build_cov(union)
    K, m = cv["K"], cv["m"]
    u = np.arange(n, n + R)
    A = np.clip(cat["A_obs"], 0.02, None)
    atil = np.log(A) + 0.02 * rng.standard_normal(n)
    sig = cat["A_sigma"] / A
    blk = np.zeros(n, dtype=np.int32)
    order = np.argsort(cat["l"])
    for k, g in enumerate(np.array_split(order, 6)):
        blk[g] = k
    groups = [np.flatnonzero(blk == k) for k in range(6)]
    blocks = [dict(Kku=K[np.ix_(g, u)], Kkk=K[np.ix_(g, g)], m=m[g], atil=atil[g],
                   sig2=sig[g] ** 2) for g in groups]
    ref_m, ref_c = P.pitc_posterior_direct(K[np.ix_(u, u)], blocks, m[u])
    cfg = gm.config_from_catalogue(cat, precision=gm.PREC_FP64, likelihood=gm.LIK_GAUSS_IN_LNA)
    with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], atil, sig) as ctx:
        ctx.build_cov()
        mean, cov = ctx.pic_posterior(blk, li, bi, si)
    np.testing.assert_allclose(mean, ref_m, rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(cov, ref_c, rtol=1e-6, atol=1e-10)


def test_pic_predict_matches_oracle(gm):
    cat = catalogue_subset(make_catalogue("c1_plain_400", truth="mean"), np.arange(300))
    n = len(cat["s"])
    rng = np.random.default_rng(9)
    R = 40
    li = rng.uniform(cat["l"].min(), cat["l"].max(), R)
    bi = rng.uniform(cat["b"].min(), cat["b"].max(), R)
    si = np.exp(rng.uniform(np.log(150), np.log(2500), R))
    jq = rng.choice(n, 20, replace=False)
    ql, qb, qs = cat["l"][jq] + 3e-4, cat["b"][jq] - 3e-4, cat["s"][jq] * 0.93
    union = dict(cat, l=np.concatenate([cat["l"], li, ql]), b=np.concatenate([cat["b"], bi, qb]),
                 s=np.concatenate([cat["s"], si, qs]))
    cv = O.build_cov(union)
    K, m = cv["K"], cv["m"]
    u = np.arange(n, n + R)
    A = np.clip(cat["A_obs"], 0.02, None)
    atil = np.log(A) + 0.02 * rng.standard_normal(n)
    sig = cat["A_sigma"] / A
    blk = np.zeros(n, dtype=np.int32)
    for k, g in enumerate(np.array_split(np.argsort(cat["l"]), 6)):
        blk[g] = k
    groups = [np.flatnonzero(blk == k) for k in range(6)]
    blocks = [dict(Kku=K[np.ix_(g, u)], Kkk=K[np.ix_(g, g)], m=m[g], atil=atil[g],
                   sig2=sig[g] ** 2) for g in groups]
    ref_m, ref_c = P.pitc_posterior_direct(K[np.ix_(u, u)], blocks, m[u])
    cfg = gm.config_from_catalogue(cat, precision=gm.PREC_FP64, likelihood=gm.LIK_GAUSS_IN_LNA)
    with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], atil, sig) as ctx:
        ctx.build_cov()
        ctx.pic_posterior(blk, li, bi, si)
        pm, pv = ctx.pic_predict(blk[jq], ql, qb, qs)
    for q in range(len(jq)):
        k = blk[jq[q]]
        j = n + R + q
        mm_, vv_ = P.pic_predict(K[np.ix_(u, u)], m[u], ref_m, ref_c, blocks[k],
                                 K[np.ix_([j], u)], np.diag(K)[[j]], K[np.ix_([j], groups[k])],
                                 m[[j]])
        assert pm[q] == pytest.approx(mm_[0], rel=1e-7, abs=1e-9)
        assert pv[q] == pytest.approx(vv_[0], rel=1e-6, abs=1e-10)
