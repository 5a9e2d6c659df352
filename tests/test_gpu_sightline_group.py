"""The grouped path of gm_predict_sightlines (m = 4, 8, 16 or 32 points per
sightline: the points of a sightline share one panel group and their cross
terms come from the m solves) on the GPU against the oracle."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("m", [8, 16])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_grouped_sightline_predictive_matches_oracle(gm, m, prec):
    cat = catalogue_subset(make_catalogue("c1_plain_400"), np.arange(200))
    cv = O.build_cov(cat)
    rng = np.random.default_rng(12)
    j = rng.choice(len(cat["s"]), 6, replace=False)
    lq, bq = cat["l"][j] + 2e-4, cat["b"][j] - 2e-4
    sq = np.sort(cat["s"][j][:, None] * np.linspace(0.4, 1.4, m)[None, :], axis=1)
    p = gm.PREC_FP64 if prec == "fp64" else gm.PREC_FP32
    cfg = gm.config_from_catalogue(cat, precision=p, cg_tol=1e-10 if prec == "fp64" else 1e-6)
    with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
        ctx.build_cov()
        ctx.ep_sweep(3, 0.0)
        tau, nu = ctx.get_sites()
        mean, cov = ctx.predict_sightlines(lq, bq, sq)
    mu_o, S_o = M.sightline_predictive(cat, cv["K"], cv["m"], tau, nu, lq, bq, sq)
    if prec == "fp64":
        np.testing.assert_allclose(mean, mu_o, rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(cov, S_o, rtol=1e-6, atol=1e-10)
    else:
        np.testing.assert_allclose(mean, mu_o, atol=1e-3)
        np.testing.assert_allclose(cov, S_o, rtol=1e-2, atol=5e-6)
