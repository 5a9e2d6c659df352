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
    CUDA-core FP32 kernel (same tolerance class), for every variant of the
    tile product (gathers one or two steps ahead, warp-specialised ring, B
    copied asynchronously from BF16 planes of PD)."""
    cat = catalogue_subset(make_catalogue("c2_plain_20k", truth="mean"), np.arange(2500))
    res = {}
    runs = [("fp64", gm.PREC_FP64, None, None), ("simt", gm.PREC_FP32, "simt", None)]
    runs += [("tc%d" % v, gm.PREC_FP32, None, str(v)) for v in (1, 2, 3, 4)]
    for name, prec, env, variant in runs:
        if env:
            monkeypatch.setenv("GM_SPMM", env)
        else:
            monkeypatch.delenv("GM_SPMM", raising=False)
        if variant:
            monkeypatch.setenv("GM_TC_PREFETCH", variant)
        else:
            monkeypatch.delenv("GM_TC_PREFETCH", raising=False)
        cfg = gm.config_from_catalogue(cat, precision=prec, probe_factor=probe,
                                       cg_tol=1e-10 if prec == gm.PREC_FP64 else 1e-6)
        with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
            ctx.build_cov()
            ctx.profile(True)
            ctx.ep_sweep(3, 0.0)
            mu, var = ctx.get_posterior()
            res[name] = (mu, var, ctx.kernel_times())
    monkeypatch.delenv("GM_SPMM", raising=False)
    monkeypatch.delenv("GM_TC_PREFETCH", raising=False)
    assert "k_panel_spmm_tiled" in res["simt"][2]
    mu64, v64 = res["fp64"][0], res["fp64"][1]
    err = {k: (np.abs(res[k][0] - mu64).max(), np.max(np.abs(res[k][1] - v64) / v64))
           for k in ("tc1", "tc2", "tc3", "tc4", "simt")}
    for v in ("tc1", "tc2", "tc3", "tc4"):
        assert "k_panel_spmm_tc" in res[v][2] and "k_panel_spmm_tiled" not in res[v][2]
        print("FP32 vs FP64 after 3 sweeps (mean, var rel): tensor cores (%s) %.2e %.2e, "
              "CUDA cores %.2e %.2e" % ((v,) + err[v] + err["simt"]))
        for k in (0, 1):
            assert err[v][k] <= 3 * err["simt"][k] + 1e-6
        assert err[v][0] < 1e-3 and err[v][1] < 1e-2
    # the variants compute the same products in the same order: equal results
    for v in ("tc2", "tc3"):
        assert np.array_equal(res[v][0], res["tc1"][0]) and np.array_equal(res[v][1], res["tc1"][1])
    # the same BF16 pieces with B read MN-major: equal up to the tensor core's
    # internal summation order
    assert "k_split3_planes" in res["tc4"][2]
    np.testing.assert_allclose(res["tc4"][0], res["tc1"][0], rtol=0, atol=1e-6)
    np.testing.assert_allclose(res["tc4"][1], res["tc1"][1], rtol=1e-5, atol=0)


def test_tile_union_and_order(gm, monkeypatch):
    """The block unions built from per-block bitmaps equal those of the sort of
    (block, column) keys (same K-steps, bit-identical posterior), and the k-d
    order of the tile rows gives fewer K-steps than the cell order with the
    same posterior to FP32 rounding."""
    cat = catalogue_subset(make_catalogue("c2_plain_20k", truth="mean"), np.arange(3000))
    out = {}
    for name, union, order in [("bitmap", None, None), ("sort", "sort", None),
                               ("rows", None, "rows")]:
        for var, val in (("GM_TC_UNION", union), ("GM_TC_ORDER", order)):
            if val:
                monkeypatch.setenv(var, val)
            else:
                monkeypatch.delenv(var, raising=False)
        cfg = gm.config_from_catalogue(cat, precision=gm.PREC_FP32, cg_tol=1e-6,
                                       probe_factor=2.0)
        with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
            ctx.build_cov()
            ctx.ep_sweep(2, 0.0)
            mu, var = ctx.get_posterior()
            out[name] = (mu, var, ctx.stats()["tile_ksteps"])
    assert out["bitmap"][2] == out["sort"][2] > 0
    np.testing.assert_array_equal(out["bitmap"][0], out["sort"][0])
    np.testing.assert_array_equal(out["bitmap"][1], out["sort"][1])
    print("tile K-steps: k-d order %d, cell order %d" % (out["bitmap"][2], out["rows"][2]))
    assert out["bitmap"][2] < out["rows"][2]
    rel = np.abs(out["bitmap"][1] - out["rows"][1]) / out["rows"][1]
    assert rel.max() < 1e-3 and np.median(rel) < 1e-5
    assert np.abs(out["bitmap"][0] - out["rows"][0]).max() < 1e-4
