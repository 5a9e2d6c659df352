"""The mixed form of the tensor-core panel product (tc_products = 3) on the
GPU against the FP32-grade form and the FP64 path."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("variant", ["1", "2", "3", "4"])
def test_mixed_form_within_the_equal_error_bar(gm, monkeypatch, variant):
    cat = catalogue_subset(make_catalogue("c2_plain_20k", truth="mean"), np.arange(2500))
    monkeypatch.setenv("GM_TC_PREFETCH", variant)
    res = {}
    for name, prec, np_ in (("fp64", gm.PREC_FP64, 6), ("fp32", gm.PREC_FP32, 6),
                            ("mixed", gm.PREC_FP32, 3)):
        cfg = gm.config_from_catalogue(cat, precision=prec, tc_products=np_,
                                       cg_tol=1e-10 if prec == gm.PREC_FP64 else 1e-6)
        with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
            ctx.build_cov()
            ctx.ep_sweep(3, 0.0)
            res[name] = ctx.get_posterior()
    mu64, v64 = res["fp64"]
    for name in ("fp32", "mixed"):
        mu, v = res[name]
        assert np.abs(mu - mu64).max() < 1e-3
        assert np.max(np.abs(v - v64) / v64) < 1e-2
