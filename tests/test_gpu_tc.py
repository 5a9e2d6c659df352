"""The tensor-core panel product of the FP32 variance solves (BF16 three-piece
split of both operands, FP32 accumulation in tensor memory) against the
CUDA-core tiled product and the FP64 path."""
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


@pytest.mark.parametrize("probe", [0.0, 2.0])
def test_tensor_core_panel_product_matches_simt_and_fp64(gm, monkeypatch, probe):
    """The tensor-core FP32 errors against the FP64 path must be those of the
    CUDA-core FP32 kernel (same tolerance class)."""
    cat = catalogue_subset(make_catalogue("c2_plain_20k", truth="mean"), np.arange(2500))
    res = {}
    for name, prec, env in (("fp64", gm.PREC_FP64, None), ("tc", gm.PREC_FP32, None),
                            ("simt", gm.PREC_FP32, "simt")):
        if env:
            monkeypatch.setenv("GM_SPMM", env)
        else:
            monkeypatch.delenv("GM_SPMM", raising=False)
        cfg = gm.config_from_catalogue(cat, precision=prec, probe_factor=probe,
                                       cg_tol=1e-10 if prec == gm.PREC_FP64 else 1e-6)
        with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
            ctx.build_cov()
            ctx.profile(True)
            ctx.ep_sweep(3, 0.0)
            mu, var = ctx.get_posterior()
            res[name] = (mu, var, ctx.kernel_times())
    monkeypatch.delenv("GM_SPMM", raising=False)
    assert "k_panel_spmm_tc" in res["tc"][2] and "k_panel_spmm_tiled" not in res["tc"][2]
    assert "k_panel_spmm_tiled" in res["simt"][2]
    mu64, v64 = res["fp64"][0], res["fp64"][1]
    err = {k: (np.abs(res[k][0] - mu64).max(), np.max(np.abs(res[k][1] - v64) / v64))
           for k in ("tc", "simt")}
    print("FP32 vs FP64 after 3 sweeps (mean, var rel): tensor cores %.2e %.2e, "
          "CUDA cores %.2e %.2e" % (err["tc"] + err["simt"]))
    for k in (0, 1):
        assert err["tc"][k] <= 3 * err["simt"][k] + 1e-6
    assert err["tc"][0] < 1e-3 and err["tc"][1] < 1e-2
