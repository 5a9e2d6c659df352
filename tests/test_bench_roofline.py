"""The roofline arithmetic of bench.py on made-up launch records: algorithmic
work per launch over the mean launch time, against the stated peak."""
import pytest

import bench


ST = {"n_stars": 20000, "nnz": 31613664, "n_pairs": 15816832, "tile_ksteps": 24990}


def test_tile_product_against_bf16_over_six():
    # 705 launches, 2183.5 ms: 3.097 ms per launch at panel width 4,640
    r = bench.roofline_for("k_panel_spmm_tc", 705, 2183.539, ST, "fp32", 4640)
    flops = 2.0 * ST["nnz"] * 4640
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(flops / (2183.539e-3 / 705) / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    peaks = bench.peaks()
    if "bf16_tflops_sustained" in peaks:
        assert r["peak"] == pytest.approx(peaks["bf16_tflops_sustained"] / 6.0)
    # executed MMA work: 6 MMAs of 2 x 128 x 16 x 256 flop per K-step and column group
    exe = ST["tile_ksteps"] * 6 * 2.0 * 128 * 16 * 256 * 19
    assert r["tensor_pipe"]["executed_tflops"] == pytest.approx(exe / (2183.539e-3 / 705) / 1e12)


def test_cuda_core_product_against_derived_fp32_peak():
    r = bench.roofline_for("k_panel_spmm_tiled", 2025, 125073.889, ST, "fp32", 20000)
    assert r["bound"] == "alu"
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2.07 / 1e3)
    assert r["achieved"] == pytest.approx(2.0 * ST["nnz"] * 20000 / (125073.889e-3 / 2025) / 1e12)


def test_sparse_matrix_vector_is_hbm_bound():
    r = bench.roofline_for("k_apply_B", 864, 160.181, ST, "fp32", 4640)
    byt = ST["nnz"] * 8 + (ST["n_stars"] + 1) * 8 + 3 * ST["n_stars"] * 4
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(byt / (160.181e-3 / 864) / 1e9)
