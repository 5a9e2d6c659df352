"""The warp-per-sightline sampler (GM_HMC_WARP=1) on the GPU against the
one-thread sampler and the oracle's chain."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("m", [2, 16, 32])
def test_warp_sampler_matches_thread_sampler_and_oracle(gm, monkeypatch, m):
    rng = np.random.default_rng(m)
    nsl, burn, ns = 1000, 10, 20
    s = np.linspace(0.0, 1.0, m)
    base = np.exp(-np.abs(s[:, None] - s[None, :]) / 0.4)
    S = (0.02 + 0.03 * rng.random(nsl))[:, None, None] * base + 1e-4 * np.eye(m)
    mu = np.cumsum(rng.normal(0.0, 0.05, (nsl, m)), axis=1) - 1.0
    mom = rng.standard_normal((nsl, burn + ns, m))
    cat = catalogue_subset(make_catalogue("c1_plain_400"), np.arange(50))
    cfg = gm.config_from_catalogue(cat)
    res = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("GM_HMC_WARP", mode)
        with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
            res[mode] = ctx.monotone_sample(mu, S, mom, burn)
    monkeypatch.delenv("GM_HMC_WARP", raising=False)
    np.testing.assert_array_equal(res["1"][1], res["0"][1])
    np.testing.assert_allclose(res["1"][0], res["0"][0], rtol=0, atol=1e-11)
    for q in rng.choice(nsl, 5, replace=False):
        ref = M.monotone_sightline(mu[q], S[q], ns, None, burn=burn, momenta=mom[q])
        np.testing.assert_allclose(res["1"][0][q], ref, rtol=0, atol=1e-9)
