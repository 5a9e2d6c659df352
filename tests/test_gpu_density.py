"""Pseudo-density on the GPU (gm_predict_pairs) against the oracle's
two-point predictive and closed-form moments (oracle/density.py)."""
import numpy as np
import pytest

import oracle as O
from oracle import density as Dn
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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pair_predictive_and_density_match_oracle(gm, prec):
    cat = catalogue_subset(make_catalogue("c1_plain_400"), np.arange(200))
    cv = O.build_cov(cat)
    rng = np.random.default_rng(3)
    j = rng.choice(len(cat["s"]), 40, replace=False)
    lq, bq = cat["l"][j] + 2e-4, cat["b"][j] - 2e-4
    sq = cat["s"][j] * rng.uniform(0.5, 1.2, len(j))
    p = gm.PREC_FP64 if prec == "fp64" else gm.PREC_FP32
    cfg = gm.config_from_catalogue(cat, precision=p, cg_tol=1e-10 if prec == "fp64" else 1e-6)
    with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
        ctx.build_cov()
        ctx.ep_sweep(3, 0.0)
        tau, nu = ctx.get_sites()
        mean, cov, dens = ctx.predict_pairs(lq, bq, sq, 10.0)
    mu_o, S_o = Dn.predict_pairs(cat, cv["K"], cv["m"], tau, nu, lq, bq, sq, 10.0)
    # the single-point predictive's parity bounds (FP64 1e-6; FP32 form 1e-3
    # in ln A and 1e-2 relative in variance)
    if prec == "fp64":
        np.testing.assert_allclose(mean, mu_o, rtol=1e-6, atol=1e-8)
        for k, (a, b_) in enumerate(((0, 0), (1, 1), (0, 1))):
            np.testing.assert_allclose(cov[:, k], S_o[:, a, b_], rtol=1e-6, atol=1e-10)
    else:
        np.testing.assert_allclose(mean, mu_o, atol=1e-3)
        for k, (a, b_) in enumerate(((0, 0), (1, 1), (0, 1))):
            np.testing.assert_allclose(cov[:, k], S_o[:, a, b_], rtol=1e-2, atol=1e-6)
    dm = np.array([Dn.density_moments(mu_o[q], S_o[q], 10.0) for q in range(len(sq))])
    print("%s pseudo-density: mean %.3e mag/pc, max rel err mean %.2e, var %.2e"
          % (prec, np.mean(dm[:, 0]), np.max(np.abs(dens[:, 0] - dm[:, 0]) / np.abs(dm[:, 0])),
             np.max(np.abs(dens[:, 1] - dm[:, 1]) / np.abs(dm[:, 1]))))
    # the density is a difference of close extinctions over 10 pc, so it
    # amplifies the predictive's errors by about s / ds
    if prec == "fp64":
        np.testing.assert_allclose(dens[:, 0], dm[:, 0], rtol=1e-4)
        np.testing.assert_allclose(dens[:, 1], dm[:, 1], rtol=1e-3)
    else:
        np.testing.assert_allclose(dens[:, 0], dm[:, 0], rtol=0.2)
        assert np.all(dens[:, 1] > 0) and np.all(np.isfinite(dens))
