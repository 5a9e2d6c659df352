"""Band-rule covariance quadrature on the GPU (quad_rule = GM_QUAD_BAND)
against the oracle's band rule (oracle/band.py) with the device constants."""
import numpy as np
import pytest

import oracle as O
from oracle import band as Bd
from synth import catalogue_subset, make_catalogue

pytestmark = pytest.mark.gpu
RULE = dict(n=6, h0=1e-3, q=3.0, m0=0.25, K=40.0)


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
def test_band_K_matches_oracle(gm, prec):
    cat = catalogue_subset(make_catalogue("c2_plain_20k", truth="mean"), np.arange(400))
    ref = Bd.build_cov_band(cat, **RULE)
    p = gm.PREC_FP64 if prec == "fp64" else gm.PREC_FP32
    cfg = gm.config_from_catalogue(cat, precision=p, quad_rule=gm.QUAD_BAND)
    with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
        ctx.build_cov()
        i, j = np.nonzero(ref["K"])
        got = ctx.get_entries(i, j)
        m, kd = ctx.get_prior()
    tol = 1e-9 if prec == "fp64" else 2e-5
    np.testing.assert_allclose(got, ref["K"][i, j], rtol=tol, atol=1e-12)
    np.testing.assert_allclose(kd, ref["diag"], rtol=tol)
    np.testing.assert_allclose(m, ref["m"], rtol=tol, atol=1e-12)
